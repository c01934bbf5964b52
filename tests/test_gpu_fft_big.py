"""GPU parity of the four-step FFT evaluator (tables beyond one CTA's shared
memory, P1 P2 > 2^14 grid points) against the FP64 oracle, through the C ABI.

The caterpillar shape at grid step 1/64 is where these tables arise: its
centroid calls have depth tables of up to ~10^7 grid units. Tolerance as in
the other parity tests: per channel, normwise, 1e-4 for FP32 fields.
"""
import numpy as np
import pytest

import workloads as W
from oracle import brute

from ._lib import tfi
from .test_gpu_parity import _stratified_targets

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4


def _err(y, ref):
    y = np.asarray(y, dtype=np.float64).reshape(ref.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return float((np.abs(y - ref).max(0) / np.maximum(np.abs(ref).max(0), 1e-300)).max())


def _apply(p, F):
    y = p.apply(torch.from_numpy(F).cuda())
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("kernel", ["cauchy", "exp", "gauss"])
@pytest.mark.parametrize("d", [1, 3, 16])
def test_caterpillar_2p14_all_outputs(kernel, d):
    # whole tables (no support truncation, which would shrink the exp and gauss tables below 2^14)
    cfg = W.configs.sweep(shape="caterpillar", n=1 << 14, d=d, kernel=kernel)
    t = cfg["tree"]
    p = tfi.Plan.from_spec(t, cfg["delta"], cfg["kernel"], leaf_max=64, max_channels=d, truncate=False)
    assert p.info()["n_jobs_fft_big"] > 0
    F = W.normal_field(t.n, d, seed=123)
    y = _apply(p, F)
    assert _err(y, brute.integrate(t, cfg["delta"], cfg["kernel"], F.astype(np.float64))) <= TOL


@pytest.mark.parametrize("d", [2, 16])
def test_two_dimensional_tables_forced(d):
    # diameter calls whose (depth x backbone) tables exceed 2^14 points, forced onto the four-step
    # evaluator: block rows and a backbone axis inside each block (N1b > 1, P2 > 1)
    cfg = W.configs.rrt_n2000()
    for t, delta, spec in [(cfg["tree"], cfg["delta"], cfg["kernel"]),
                           (W.toothed_spine(2000, 3), 1.0, W.KernelSpec.exp(0.01))]:
        p = tfi.Plan.from_spec(t, delta, spec, policy="diameter", leaf_max=1, max_channels=d, fft_big_all=True)
        jobs = p.export("jobs")
        assert (jobs[:, 0] == 4).any()
        F = W.normal_field(t.n, d, seed=9)
        assert _err(_apply(p, F), brute.integrate(t, delta, spec, F.astype(np.float64))) <= TOL


def test_caterpillar_2p19_stratified_batches_and_adjoint():
    # tables of up to 2^24 points (columns of 2^12, the two-column pass), several buffer batches
    # at d = 16; sampled outputs including members of every four-step size class
    cfg = W.configs.sweep(shape="caterpillar", n=1 << 19, d=16, kernel="cauchy")
    t = cfg["tree"]
    p = tfi.Plan.from_spec(t, cfg["delta"], cfg["kernel"], leaf_max=512, max_channels=16)
    jobs = p.export("jobs")
    big = jobs[jobs[:, 0] == 4]
    assert len(big) > 0 and big[:, 1].max() >= 24
    targets, _ = _stratified_targets(p, t.n, seed=2, per=48, n_random=96)
    extra = []
    for lnp in np.unique(big[:, 1]):
        sel = big[big[:, 1] == lnp][:8]
        extra += list(sel[:, 4]) + list(sel[:, 5])
    targets = np.unique(np.concatenate([targets, np.asarray(extra, dtype=np.int32)])).astype(np.int32)
    F = W.normal_field(t.n, 16, seed=123)
    x = torch.from_numpy(F).cuda()
    y1 = p.apply(x)
    y2 = p.apply(x)
    assert torch.equal(y1, y2)
    ref = brute.integrate(t, cfg["delta"], cfg["kernel"], F.astype(np.float64), targets=targets)
    assert _err(y1.cpu().numpy()[targets], ref) <= TOL
    z = torch.randn_like(x)
    lhs = float((z.double() * y1.double()).sum())
    rhs = float((p.apply_backward(z).double() * x.double()).sum())
    assert abs(lhs - rhs) <= 1e-4 * (abs(lhs) + abs(rhs) + 1.0)


def test_graph_replay_with_big_tables():
    cfg = W.configs.sweep(shape="caterpillar", n=1 << 14, d=8, kernel="exp")
    t = cfg["tree"]
    p = tfi.Plan.from_spec(t, cfg["delta"], cfg["kernel"], leaf_max=64, max_channels=8, truncate=False)
    assert p.info()["n_jobs_fft_big"] > 0
    x = torch.from_numpy(W.normal_field(t.n, 8, seed=3)).cuda()
    z = torch.from_numpy(W.normal_field(t.n, 8, seed=4)).cuda()
    out, gF = torch.empty_like(x), torch.empty_like(x)
    g = tfi.Graph(p, x, out, z, gF)
    g.launch()
    torch.cuda.synchronize()
    assert torch.equal(out, p.apply(x)) and torch.equal(gF, p.apply(z))
