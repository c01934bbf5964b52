"""Exponential-sum sweeps (Algorithm 7) as the table evaluator (TFI_PLAN_SWEEP),
through the C ABI, against the FP64 oracle."""
import numpy as np
import pytest

import workloads as W
from oracle import brute

from ._lib import tfi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _err(y, ref):
    y = np.asarray(y, dtype=np.float64).reshape(ref.shape[0], -1)
    return float((np.abs(y - ref).max(0) / np.maximum(np.abs(ref).max(0), 1e-300)).max())


def _check(t, delta, spec, d, policy="adaptive", leaf_max=64, tol=1e-4, targets=None):
    p = tfi.Plan.from_spec(t, delta, spec, policy=policy, leaf_max=leaf_max, max_channels=d, sweep=True)
    info = p.info()
    assert info["n_jobs_fft"] == 0 and info["n_jobs_direct"] == 0 and info["n_jobs_sweep"] >= info["n_calls"]
    F = W.normal_field(t.n, d, seed=17)
    y = p.apply(torch.from_numpy(F).cuda()).cpu().numpy()
    ref = brute.integrate(t, delta, spec, F.astype(np.float64), targets=targets)
    if targets is not None:
        y = y[targets]
    assert _err(y, ref) <= tol
    return p


@pytest.mark.parametrize("policy", ["adaptive", "diameter", "centroid"])
@pytest.mark.parametrize("leaf_max", [1, 64])
def test_sweep_rrt_n2000(policy, leaf_max):
    cfg = W.configs.rrt_n2000()
    _check(cfg["tree"], cfg["delta"], cfg["kernel"], 16, policy=policy, leaf_max=leaf_max)


def test_sweep_grid_weights_and_long_path():
    cfg = W.configs.sweep(shape="caterpillar", n=4096, d=4, kernel="exp")
    _check(cfg["tree"], cfg["delta"], cfg["kernel"], 4)
    path = W.path(5000).with_weights(np.random.default_rng(1).integers(1, 9, 4999) / 8.0)
    _check(path, 1 / 8, W.KernelSpec.exp(0.3), 3, policy="diameter", leaf_max=1)


def test_sweep_expsum_attention_trees():
    cfg = W.configs.attention(heads=2)
    for h in cfg["heads"]:
        _check(h["tree"], 1.0, h["kernel"], 64, leaf_max=16)


def test_sweep_full_size_sampled():
    cfg = W.configs.sweep(shape="rrt", n=1 << 20, d=16, kernel="exp")
    tgt = np.sort(np.random.default_rng(2).choice(cfg["tree"].n, 32, replace=False)).astype(np.int32)
    _check(cfg["tree"], cfg["delta"], cfg["kernel"], 16, leaf_max=512, targets=tgt)


def test_sweep_requires_expsum():
    t = W.path(10)
    with pytest.raises(tfi.TfiError):
        tfi.Plan.from_spec(t, 1.0, W.KernelSpec.gauss(0.1), sweep=True)


@pytest.mark.parametrize("make,delta,policy,d", [
    (lambda: W.configs.sweep("rrt", n=1 << 15, d=16)["tree"], 1 / 64, "adaptive", 16),
    (lambda: W.configs.sweep("caterpillar", n=1 << 12, d=16)["tree"], 1 / 64, "diameter", 16),
    (lambda: W.configs.rrt_n2000()["tree"], 1.0, "diameter", 20),
    (lambda: W.spider(6, 300), 1.0, "adaptive", 33),
])
def test_sweep_auto_mixed_evaluators(make, delta, policy, d):
    # TFI_PLAN_SWEEP_AUTO: per table the cheaper of sweeps and FFT / direct; plans mix the modes
    t = make()
    spec = W.KernelSpec.expsum([1.0, -0.3], [0.1, 0.7])
    p = tfi.Plan.from_spec(t, delta, spec, policy=policy, leaf_max=16, max_channels=d, sweep="auto")
    info = p.info()
    assert info["n_jobs_sweep"] > 0  # the large trees also keep small tables on FFT / direct
    F = W.normal_field(t.n, d, seed=19)
    y = p.apply(torch.from_numpy(F).cuda()).cpu().numpy()
    rng = np.random.default_rng(2)
    targets = np.sort(rng.choice(t.n, size=min(t.n, 300), replace=False)).astype(np.int32)
    ref = brute.integrate(t, delta, spec, F.astype(np.float64), targets=targets)
    assert _err(y[targets], ref) <= 1e-4
    # the same operator as the plan without sweeps, up to rounding
    q = tfi.Plan.from_spec(t, delta, spec, policy=policy, leaf_max=16, max_channels=d)
    assert q.info()["n_jobs_sweep"] == 0
    y2 = q.apply(torch.from_numpy(F).cuda()).cpu().numpy()
    assert _err(y2[targets], ref) <= 1e-4


def test_sweep_auto_plan_in_a_cuda_graph():
    # a captured fwd+bwd step of a mixed sweep / FFT / direct plan equals the eager applies
    cfg = W.configs.sweep("rrt", n=1 << 14, d=16)
    t = cfg["tree"]
    p = tfi.Plan.from_spec(t, cfg["delta"], cfg["kernel"], leaf_max=64, max_channels=16, sweep="auto")
    assert p.info()["n_jobs_sweep"] > 0
    F = torch.from_numpy(W.normal_field(t.n, 16, seed=61)).cuda()
    G = torch.from_numpy(W.normal_field(t.n, 16, seed=62)).cuda()
    out, gF = torch.empty_like(F), torch.empty_like(F)
    g = tfi.Graph(p, F, out, G, gF)
    for _ in range(2):
        g.launch()
    torch.cuda.synchronize()
    assert torch.equal(out, p.apply(F)) and torch.equal(gF, p.apply(G))
