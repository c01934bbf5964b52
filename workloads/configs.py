"""The five benchmark workloads, as seeded generator recipes.

Each builder returns a dict with the forest (``tree``), the grid step
``delta``, the kernel spec ``kernel``, channel count ``d`` and field dtype.
Sizes can be overridden so the same recipe yields small parity cases.

* ``rrt_n2000``      random recursive tree, N=2000, integer weights {1..4},
                     d=16, f(x)=exp(-0.5x), grid step 1 (tree seed 0).
* ``sweep``          single trees of shape rrt | caterpillar | binary,
                     N in {2^14..2^20}, weights U[0.5,2] snapped to 1/64,
                     grid step 1/64, d in {1,16,64}, f in {exp(-0.1x),
                     1/(1+x^2), exp(-x^2/8)}.
* ``torus_sinkhorn`` 50,000 torus points, kNN(8) MST, grid step 1/256,
                     d=8 Dirichlet(1) marginals, f(x)=exp(-x/0.05).
* ``attention``      12 spanning trees of the 14x14 grid (one per head),
                     unit weights, d=64*64 channels, learnable
                     f = sum_{k<=8} a_k exp(-b_k x).
* ``uneven_batch``   4096 random recursive trees, sizes log-uniform in
                     [64, 65536], integer weights {1..8}, d=16,
                     f(x)=1/(1+0.1x)^2.
"""
from __future__ import annotations

import numpy as np

from . import trees as T
from .kernels import KernelSpec

SWEEP_KERNELS = {
    "exp": KernelSpec.exp(0.1),
    "cauchy": KernelSpec.rational(1.0, e=2.0, p=1.0),
    "gauss": KernelSpec.gauss(1.0 / 8.0),
}


def rrt_n2000(n: int = 2000, d: int = 16, seed: int = 0):
    rng = np.random.default_rng(seed)
    t = T.random_recursive(n, rng)
    t = t.with_weights(T.integer_weights(t.m, 1, 4, rng))
    return dict(name="rrt_n2000", tree=t, delta=1.0, kernel=KernelSpec.exp(0.5), d=d, dtype="f32")


def sweep(shape: str = "rrt", n: int = 1 << 20, d: int = 16, kernel: str = "exp", seed: int = 0):
    rng = np.random.default_rng(seed)
    if shape == "rrt":
        t = T.random_recursive(n, rng)
    elif shape == "caterpillar":
        t = T.caterpillar_rrt(n, rng)
    elif shape == "binary":
        t = T.complete_binary_n(n)
    else:
        raise ValueError(shape)
    t = t.with_weights(T.snapped_uniform_weights(t.m, 0.5, 2.0, 1.0 / 64, rng))
    return dict(name=f"sweep_{shape}", tree=t, delta=1.0 / 64, kernel=SWEEP_KERNELS[kernel], d=d, dtype="f32")


def torus_sinkhorn(n: int = 50_000, pairs: int = 8, seed: int = 0):
    rng = np.random.default_rng(seed)
    t = T.torus_knn_mst(n, rng)
    return dict(name="torus_sinkhorn", tree=t, delta=1.0 / 256, kernel=KernelSpec.exp(1.0 / 0.05), d=pairs,
                dtype="f32", iterations=200)


def attention(heads: int = 12, side: int = 14, images: int = 64, dh: int = 64, seed: int = 0):
    rng = np.random.default_rng(seed)
    heads_out = []
    for _ in range(heads):
        t = T.grid_spanning_tree(side, side, rng)
        a = rng.normal(0.0, 0.1, size=8)
        b = rng.uniform(0.1, 2.0, size=8)
        heads_out.append(dict(tree=t, a=a, b=b, kernel=KernelSpec.expsum(a, b)))
    return dict(name="attention", heads=heads_out, delta=1.0, d=images * dh, dtype="bf16")


def uneven_batch(count: int = 4096, lo: int = 64, hi: int = 65536, d: int = 16, seed: int = 0):
    rng = np.random.default_rng(seed)
    sizes = np.round(np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int64)
    ts = []
    for s in sizes:
        t = T.random_recursive(int(s), rng)
        ts.append(t.with_weights(T.integer_weights(t.m, 1, 8, rng)))
    f, offs = T.forest(ts)
    return dict(name="uneven_batch", tree=f, offsets=offs, sizes=sizes, delta=1.0,
                kernel=KernelSpec.rational(0.1, e=1.0, p=2.0), d=d, dtype="f32")
