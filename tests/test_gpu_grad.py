"""Gradient with respect to the kernel (learnable f), through the C ABI,
against the FP64 oracle's distance-binned correlation and its parameter
gradient (itself pinned by finite differences in the oracle tests)."""
import numpy as np
import pytest

import workloads as W
from oracle import brute

from ._lib import tfi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _nerr(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _grad_case(t, delta, spec, d, leaf_max, policy="adaptive", dtype=torch.float32, tol=1e-4):
    p = tfi.Plan.from_spec(t, delta, spec, policy=policy, leaf_max=leaf_max, max_channels=d)
    G = torch.from_numpy(W.normal_field(t.n, d, seed=31)).cuda().to(dtype)
    F = torch.from_numpy(W.normal_field(t.n, d, seed=32)).cuda().to(dtype)
    C, dth = p.kernel_grad(G, F)
    Gn, Fn = G.double().cpu().numpy(), F.double().cpu().numpy()
    ref = brute.corr_hist(t, delta, Gn, Fn)
    c = C.cpu().numpy()
    # the plan's histogram may extend past the largest pair distance (those bins hold only round-off)
    assert len(c) >= len(ref)
    ref = np.concatenate([ref, np.zeros(len(c) - len(ref))])
    assert _nerr(c, ref) <= tol
    if spec.kind != "table":
        assert _nerr(dth, brute.kernel_param_grad(t, delta, spec, Gn, Fn)) <= tol
    return p


@pytest.mark.parametrize("leaf_max", [1, 16, 256])
@pytest.mark.parametrize("policy", ["adaptive", "centroid"])
def test_grad_rrt_n2000(leaf_max, policy):
    cfg = W.configs.rrt_n2000()
    _grad_case(cfg["tree"], cfg["delta"], W.KernelSpec.expsum([0.5, -0.2], [0.3, 0.05]), 16, leaf_max, policy)


def test_grad_attention_heads_fp32_and_bf16():
    cfg = W.configs.attention(heads=2)
    for h in cfg["heads"]:
        _grad_case(h["tree"], 1.0, h["kernel"], 64, 256)
        _grad_case(h["tree"], 1.0, h["kernel"], 64, 16, dtype=torch.bfloat16, tol=1e-2)


def test_grad_weighted_grid_forest():
    cfg = W.configs.uneven_batch(count=10, lo=20, hi=800, d=8)
    _grad_case(cfg["tree"], cfg["delta"], W.KernelSpec.rational(0.1, e=1.0, p=2.0), 8, 32)


@pytest.mark.parametrize("spec", [
    W.KernelSpec.gauss(0.02, a=1.2),
    W.KernelSpec.rational(0.1, e=1.5, p=2.0, a=0.9),
    W.KernelSpec.powexp(0.2, p=1.3, a=1.1),
], ids=["gauss", "rational", "powexp"])
@pytest.mark.parametrize("leaf_max", [1, 32])
def test_grad_dtheta_every_analytic_kind(spec, leaf_max):
    # dL/dtheta of the gauss, rational and powexp kinds (each parameter, including the exponents
    # whose derivatives carry ln x) against the oracle's analytic derivatives, themselves pinned by
    # finite differences of the brute force
    cfg = W.configs.uneven_batch(count=6, lo=20, hi=600, d=8)
    _grad_case(cfg["tree"], 1.0, spec, 8, leaf_max)


@pytest.mark.parametrize("leaf_max", [1, 16])
def test_grad_diameter_policy_tables_beyond_one_transform(leaf_max):
    # C1 under the diameter policy: its top diameter call has a table of 2^15 grid points, beyond one
    # shared-memory transform, whose pair histogram is taken by the direct correlation
    cfg = W.configs.rrt_n2000()
    _grad_case(cfg["tree"], cfg["delta"], W.KernelSpec.expsum([0.7, -0.3], [0.4, 0.1]), 8, leaf_max,
               policy="diameter")


def test_grad_rejects_huge_tables_with_many_bins():
    # the 2^14-vertex caterpillar at grid 1/64: tables of up to 2^19 points with tens of thousands of bins
    cfg = W.configs.sweep(shape="caterpillar", n=1 << 14, d=4, kernel="exp")
    p = tfi.Plan.from_spec(cfg["tree"], cfg["delta"], cfg["kernel"], leaf_max=64, max_channels=4)
    x = torch.zeros(cfg["tree"].n, 4, device="cuda")
    with pytest.raises(tfi.TfiError) as e:
        p.kernel_grad(x, torch.zeros_like(x))
    assert e.value.name == "UNSUPPORTED"


def test_set_kernel_and_learnable_autograd():
    cfg = W.configs.attention(heads=1)
    h = cfg["heads"][0]
    t = h["tree"]
    p = tfi.Plan.from_spec(t, 1.0, h["kernel"], leaf_max=64, max_channels=32)
    theta = torch.tensor(h["kernel"].params, dtype=torch.float64, requires_grad=True)
    F = torch.from_numpy(W.normal_field(t.n, 32, seed=5)).cuda().requires_grad_(True)
    y = tfi.integrate_learnable(F, theta, p)
    g = torch.from_numpy(W.normal_field(t.n, 32, seed=6)).cuda()
    (y * g).sum().backward()
    spec = W.KernelSpec("expsum", list(h["kernel"].params))
    Fn, gn = F.detach().double().cpu().numpy(), g.double().cpu().numpy()
    assert _nerr(theta.grad.numpy(), brute.kernel_param_grad(t, 1.0, spec, gn, Fn)) <= 1e-4
    assert _nerr(F.grad.cpu().numpy(), brute.integrate(t, 1.0, spec, gn)) <= 1e-4
    # a new kernel without replanning
    new = list(h["kernel"].params)
    new[0] *= -2.0
    new[3] *= 1.5
    p.set_kernel(params=new)
    y2 = p.apply(F.detach()).cpu().numpy()
    assert _nerr(y2, brute.integrate(t, 1.0, W.KernelSpec("expsum", new), Fn)) <= 1e-4


@pytest.mark.parametrize("d,dtype,tol", [(100, torch.float32, 1e-4), (256, torch.bfloat16, 1e-4)])
def test_grad_many_channel_blocks(d, dtype, tol):
    # channels are split over CTAs in blocks of 32 and the blocks' histograms added in order:
    # a ragged last block (d = 100) and the attention trees' width class (bf16, d = 256)
    cfg = W.configs.attention(heads=1)
    h = cfg["heads"][0]
    p = _grad_case(h["tree"], 1.0, h["kernel"], d, 1, dtype=dtype, tol=tol)
    # a later call with fewer channels ignores the blocks of the wider call
    G = torch.from_numpy(W.normal_field(h["tree"].n, 8, seed=41)).cuda().to(dtype)
    F = torch.from_numpy(W.normal_field(h["tree"].n, 8, seed=42)).cuda().to(dtype)
    C, _ = p.kernel_grad(G, F)
    ref = brute.corr_hist(h["tree"], 1.0, G.double().cpu().numpy(), F.double().cpu().numpy())
    c = C.cpu().numpy()
    ref = np.concatenate([ref, np.zeros(len(c) - len(ref))])
    assert _nerr(c, ref) <= tol


def test_grad_device_dtheta_on_a_side_stream():
    # dtheta left on the device (no synchronisation) equals the host copy
    cfg = W.configs.attention(heads=1)
    h = cfg["heads"][0]
    p = tfi.Plan.from_spec(h["tree"], 1.0, h["kernel"], leaf_max=4, max_channels=64)
    G = torch.from_numpy(W.normal_field(h["tree"].n, 64, seed=51)).cuda()
    F = torch.from_numpy(W.normal_field(h["tree"].n, 64, seed=52)).cuda()
    C0, th0 = p.kernel_grad(G, F)
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    C1, th1 = p.kernel_grad(G, F, stream=st, device_dtheta=True)
    torch.cuda.current_stream().wait_stream(st)
    torch.cuda.synchronize()
    assert th1.is_cuda and np.array_equal(th1.cpu().numpy(), th0)
    assert torch.equal(C0, C1)


@pytest.mark.parametrize("leaf_max", [512, 1024])
def test_grad_large_leaves_deterministic(leaf_max):
    # leaves of hundreds of vertices (the one-pass leaf histograms: 64-bit fixed-point sums, exact
    # whatever the order of the atomic adds): oracle parity, and bit-identical repeated calls
    cfg = W.configs.sweep(shape="rrt", n=8192, d=16, kernel="exp")
    t = cfg["tree"]
    p = _grad_case(t, cfg["delta"], cfg["kernel"], 16, leaf_max)
    assert p.info()["sum_leaf_pairs"] > 1_000_000
    G = torch.from_numpy(W.normal_field(t.n, 16, seed=31)).cuda()
    F = torch.from_numpy(W.normal_field(t.n, 16, seed=32)).cuda()
    C1, _ = p.kernel_grad(G, F)
    C2, _ = p.kernel_grad(G, F)
    assert torch.equal(C1, C2)


@pytest.mark.parametrize("scale", [1e-18, 1e18])
def test_grad_leaf_histograms_follow_the_field_scale(scale):
    # the fixed-point scale adapts to each leaf's field norms: tiny and huge fields keep the bound
    cfg = W.configs.rrt_n2000()
    t = cfg["tree"]
    p = tfi.Plan.from_spec(t, cfg["delta"], cfg["kernel"], leaf_max=256, max_channels=8)
    G = torch.from_numpy((W.normal_field(t.n, 8, seed=33) * np.sqrt(scale)).astype(np.float32)).cuda()
    F = torch.from_numpy((W.normal_field(t.n, 8, seed=34) * np.sqrt(scale)).astype(np.float32)).cuda()
    C, _ = p.kernel_grad(G, F)
    ref = brute.corr_hist(t, cfg["delta"], G.double().cpu().numpy(), F.double().cpu().numpy())
    c = C.cpu().numpy()
    ref = np.concatenate([ref, np.zeros(len(c) - len(ref))])
    assert _nerr(c, ref) <= 1e-4


@pytest.mark.parametrize("dtype,tol", [(torch.float32, 1e-4), (torch.bfloat16, 1e-4)])
def test_grad_few_leaves_many_channels(dtype, tol):
    # a few big leaves and many channel blocks: the blocks spread over CTAs whose exact integer sums
    # are merged in global memory (same result whatever the split)
    rng = np.random.default_rng(41)
    t = W.random_recursive(700, rng)
    t = t.with_weights(W.trees.integer_weights(t.m, 1, 4, rng))
    for d in (48, 200):
        p = _grad_case(t, 1.0, W.KernelSpec.exp(0.05), d, 1024, dtype=dtype, tol=tol)
        assert p.info()["n_calls"] == 0   # the whole tree is one leaf
        G = torch.from_numpy(W.normal_field(t.n, d, seed=31)).cuda().to(dtype)
        F = torch.from_numpy(W.normal_field(t.n, d, seed=32)).cuda().to(dtype)
        assert torch.equal(p.kernel_grad(G, F)[0], p.kernel_grad(G, F)[0])
