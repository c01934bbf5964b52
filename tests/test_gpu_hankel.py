"""GPU parity of the Hankel-matrix evaluator (tcgen05) against the FP64 oracle.

The evaluator computes each qualifying cross table / correction as one product
with the Hankel matrix f(l + r) followed by prefix sums along antidiagonals
(attention-width evaluation of Eq. "sumofFFTterms"). Tolerance as in the other
parity tests: per channel, normwise, 1e-4 for FP32 fields and 1e-2 for BF16.
"""
import numpy as np
import pytest

import workloads as W
from oracle import brute

from ._lib import tfi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-4, "bf16": 1e-2}


def _err(y, ref):
    y = np.asarray(y, dtype=np.float64).reshape(ref.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return float((np.abs(y - ref).max(0) / np.maximum(np.abs(ref).max(0), 1e-300)).max())


def _check(t, delta, spec, F, dtype="f32", hankel="all", **kw):
    p = tfi.Plan.from_spec(t, delta, spec, max_channels=F.shape[1], hankel=hankel, **kw)
    info = p.info()
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    Fd = torch.from_numpy(F).to("cuda", tdt)
    y = p.apply(Fd)
    torch.cuda.synchronize()
    ref = brute.integrate(t, delta, spec, Fd.float().cpu().numpy().astype(np.float64))
    assert p.info()["device_errors"] == 0
    return p, info, _err(y.float().cpu().numpy(), ref)


@pytest.mark.parametrize("leaf_max", [1, 16])
@pytest.mark.parametrize("dtype,d", [("f32", 64), ("f32", 200), ("bf16", 256)])
def test_attention_grid_trees(leaf_max, dtype, d):
    cfg = W.configs.attention(heads=2)
    for h in cfg["heads"]:
        F = W.normal_field(h["tree"].n, d, seed=11)
        _, info, e = _check(h["tree"], 1.0, h["kernel"], F, dtype=dtype, leaf_max=leaf_max)
        assert info["n_jobs_hankel"] > 0
        assert e <= TOL[dtype]


@pytest.mark.parametrize("policy", ["adaptive", "diameter", "centroid"])
def test_rrt_mixed_evaluators(policy):
    # grid-unit tables beyond the Hankel limits stay on the FFT / direct evaluators in the same plan
    cfg = W.configs.rrt_n2000()
    F = W.normal_field(cfg["tree"].n, 16, seed=123)
    _, info, e = _check(cfg["tree"], cfg["delta"], cfg["kernel"], F, policy=policy, leaf_max=4)
    assert info["n_jobs_hankel"] > 0
    assert e <= TOL["f32"]


@pytest.mark.parametrize("d", [1, 3, 129])
def test_long_paths_and_ragged_channels(d):
    # a path under the diameter policy: H = 0, backbone up to 127 grid units (the row limit)
    t = W.path(128)
    F = W.normal_field(t.n, d, seed=5)
    _, info, e = _check(t, 1.0, W.KernelSpec.rational(0.3, e=1.0, p=1.5), F, policy="diameter", leaf_max=1)
    assert info["n_jobs_hankel"] >= 1
    assert e <= TOL["f32"]
    # a spider: long centroid depths (H up to 63) and many short components
    t = W.spider(6, 60)
    F = W.normal_field(t.n, d, seed=6)
    _, info, e = _check(t, 1.0, W.KernelSpec.exp(0.05), F, policy="centroid", leaf_max=2)
    assert e <= TOL["f32"]


def test_growing_kernel():
    # the appendix also checks growing kernels; FP32 stays within the normwise bound
    rng = np.random.default_rng(3)
    t = W.grid_spanning_tree(10, 10, rng)
    F = W.normal_field(t.n, 32, seed=7)
    _, info, e = _check(t, 1.0, W.KernelSpec.expsum([1.0], [-0.02]), F, leaf_max=4)
    assert info["n_jobs_hankel"] > 0 and e <= TOL["f32"]


def test_auto_selection_and_determinism():
    cfg = W.configs.attention(heads=1)
    h = cfg["heads"][0]
    mk = lambda mode: tfi.Plan.from_spec(h["tree"], 1.0, h["kernel"], leaf_max=4, max_channels=4096, hankel=mode)
    p, auto, q = mk("all"), mk("auto"), mk(None)
    assert p.info()["n_jobs_hankel"] > 0 and q.info()["n_jobs_hankel"] == 0
    assert auto.info()["n_jobs_hankel"] <= p.info()["n_jobs_hankel"]
    x = torch.randn(h["tree"].n, 4096, device="cuda", dtype=torch.bfloat16)
    y1, y2 = p.apply(x), p.apply(x)
    assert torch.equal(y1, y2)
    # every evaluator choice against the FP64 oracle on the BF16-rounded input
    ref = brute.integrate(h["tree"], 1.0, h["kernel"], x.double().cpu().numpy())
    for y in (y1, auto.apply(x), q.apply(x)):
        assert _err(y.double().cpu().numpy(), ref) <= TOL["bf16"]


def test_adjoint_graph_and_kernel_grad():
    rng = np.random.default_rng(9)
    t = W.grid_spanning_tree(9, 9, rng)
    spec = W.KernelSpec.expsum([0.5, -0.2], [0.3, 0.9])
    p = tfi.Plan.from_spec(t, 1.0, spec, leaf_max=4, max_channels=8, hankel="all")
    x = torch.randn(t.n, 8, device="cuda")
    z = torch.randn(t.n, 8, device="cuda")
    lhs = float((z.double() * p.apply(x).double()).sum())
    rhs = float((p.apply_backward(z).double() * x.double()).sum())
    assert abs(lhs - rhs) <= 1e-4 * (abs(lhs) + abs(rhs) + 1.0)
    out, gF = torch.empty_like(x), torch.empty_like(x)
    g = tfi.Graph(p, x, out, z, gF)
    g.launch()
    torch.cuda.synchronize()
    assert torch.equal(out, p.apply(x)) and torch.equal(gF, p.apply(z))
    _, dth = p.kernel_grad(z, x)
    ref = brute.kernel_param_grad(t, 1.0, spec, z.cpu().double().numpy(), x.cpu().double().numpy())
    assert np.abs(np.asarray(dth) - ref).max() <= 1e-4 * np.abs(ref).max()
