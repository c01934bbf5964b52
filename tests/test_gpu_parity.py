"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerance (per channel, normwise): max_u |y_gpu - y| / max_u |y| <= 1e-4 for
FP32 fields and <= 1e-2 for BF16 fields (the bf16 case compares against the
oracle applied to the bf16-rounded input).
"""
import ctypes

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
    scale = np.maximum(np.abs(ref).max(axis=0), 1e-300)
    return float((np.abs(y - ref).max(axis=0) / scale).max())


def _run(t, delta, spec, F, policy="adaptive", leaf_max=64, dtype="f32", targets=None):
    p = tfi.Plan.from_spec(t, delta, spec, policy=policy, leaf_max=leaf_max, max_channels=F.shape[1])
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    Fd = torch.from_numpy(F).to("cuda", tdt)
    y = p.apply(Fd)
    torch.cuda.synchronize()
    Fin = Fd.float().cpu().numpy().astype(np.float64)
    ref = brute.integrate(t, delta, spec, Fin, targets=targets)
    yv = y.float().cpu().numpy()
    if targets is not None:
        yv = yv[targets]
    return p, yv, ref


def _rrt(n, seed, lo=1, hi=4):
    rng = np.random.default_rng(seed)
    t = W.random_recursive(n, rng)
    return t.with_weights(W.trees.integer_weights(t.m, lo, hi, rng))


@pytest.mark.parametrize("policy", ["adaptive", "diameter", "centroid"])
@pytest.mark.parametrize("leaf_max", [1, 16, 64, 256])
def test_rrt_n2000_config(policy, leaf_max):
    cfg = W.configs.rrt_n2000()
    F = W.normal_field(cfg["tree"].n, cfg["d"], seed=123)
    _, y, ref = _run(cfg["tree"], cfg["delta"], cfg["kernel"], F, policy=policy, leaf_max=leaf_max)
    assert _err(y, ref) <= TOL["f32"]


@pytest.mark.parametrize("shape", ["rrt", "binary", "caterpillar"])
@pytest.mark.parametrize("kernel", ["exp", "cauchy", "gauss"])
@pytest.mark.parametrize("d", [1, 16, 64])
def test_sweep_shapes_small(shape, kernel, d):
    cfg = W.configs.sweep(shape=shape, n=4096 if shape != "caterpillar" else 2048, d=d, kernel=kernel)
    F = W.normal_field(cfg["tree"].n, d, seed=123)
    _, y, ref = _run(cfg["tree"], cfg["delta"], cfg["kernel"], F, leaf_max=64)
    assert _err(y, ref) <= TOL["f32"]


@pytest.mark.parametrize("make", [lambda: W.spider(8, 200), lambda: W.caterpillar_hanging_paths(24),
                                  lambda: W.path(3000), lambda: W.star(500), lambda: W.complete_kary(3, 6),
                                  lambda: W.caterpillar_leaves(300), lambda: W.broom(400),
                                  lambda: W.preferential_attachment(3000, np.random.default_rng(3))])
@pytest.mark.parametrize("policy", ["adaptive", "diameter"])
def test_paper_families_unit_weights(make, policy):
    t = make()
    F = W.normal_field(t.n, 3, seed=7)
    _, y, ref = _run(t, 1.0, W.KernelSpec.rational(1.0), F, policy=policy, leaf_max=8)
    assert _err(y, ref) <= TOL["f32"]


@pytest.mark.parametrize("make", [lambda: W.spider(8, 60), lambda: W.spider(8, 100),
                                  lambda: W.toothed_spine(200, 2), lambda: W.toothed_spine(256, 3)],
                         ids=["1d_2^7", "1d_2^8", "2d_2^3x2^9", "2d_2^3x2^10"])
@pytest.mark.parametrize("d", [3, 8, 16])
def test_fft_table_shapes(make, d):
    # FFT tables the larger workloads do not produce: one-dimensional tables of 2^7 and 2^8
    # points (radix-2 / radix-4 first passes) and two-dimensional ones (the general passes of the
    # two-pair kernel, and the one-pair kernel at 2^13 points), at 2, 4 and 8 channel pairs
    t = make()
    F = W.normal_field(t.n, d, seed=5)
    p, y, ref = _run(t, 1.0, W.KernelSpec.exp(0.05), F, leaf_max=8)
    assert p.info()["n_jobs_fft"] > 0
    assert _err(y, ref) <= TOL["f32"]


def test_forest_uneven_batch_small():
    cfg = W.configs.uneven_batch(count=40, lo=8, hi=3000, d=16)
    F = W.normal_field(cfg["tree"].n, 16, seed=123)
    _, y, ref = _run(cfg["tree"], cfg["delta"], cfg["kernel"], F, leaf_max=64)
    assert _err(y, ref) <= TOL["f32"]


def test_torus_mst_small():
    cfg = W.configs.torus_sinkhorn(n=4000, pairs=8)
    a, _ = W.dirichlet_pairs(cfg["tree"].n, 8, seed=1)
    _, y, ref = _run(cfg["tree"], cfg["delta"], cfg["kernel"], a.astype(np.float32), leaf_max=64)
    assert _err(y, ref) <= TOL["f32"]


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_attention_grid_trees(dtype):
    cfg = W.configs.attention(heads=2)
    for h in cfg["heads"]:
        F = W.normal_field(h["tree"].n, 64, seed=11)
        _, y, ref = _run(h["tree"], 1.0, h["kernel"], F, leaf_max=64, dtype=dtype)
        assert _err(y, ref) <= TOL[dtype]


def _stratified_targets(p, n, seed, per=96, n_random=128):
    """Target vertices that reach every part of a plan: backbone vertices of the top two
    recursion levels, the deepest records, the smallest vertex of the largest dense leaves,
    member vertices of tables of every FFT size class and of direct tables, and uniform ones."""
    rng = np.random.default_rng(seed)
    calls, bb = p.export("calls"), p.export("backbone")
    off = np.concatenate([[0], np.cumsum(calls[:, 4])])
    top = np.concatenate([bb[off[i]:off[i + 1]] for i in np.nonzero(calls[:, 0] <= 1)[0]])
    picks = [top[:per]]
    recs = p.export("records")
    picks.append(recs[np.argsort(-recs[:, 2], kind="stable")[:per], 1])
    del recs
    leaves = p.export("leaves")
    picks.append(leaves[np.argsort(-leaves[:, 2], kind="stable")[:per], 1])
    jobs = p.export("jobs")
    classes = np.unique(jobs[jobs[:, 0] == 0, 1])
    for lnp in classes:
        sel = jobs[(jobs[:, 0] == 0) & (jobs[:, 1] == lnp)]
        sel = sel[rng.permutation(len(sel))[:16]]
        picks += [sel[:, 4], sel[:, 5]]
    sel = jobs[jobs[:, 0] == 1]
    sel = sel[rng.permutation(len(sel))[:32]]
    picks += [sel[:, 4], sel[:, 5]]
    picks.append(rng.choice(n, n_random, replace=False))
    t = np.unique(np.concatenate(picks))
    return t[t >= 0].astype(np.int32), len(classes)


def _full_size_case(shape, n, leaf_max, per, n_random, min_targets, **flags):
    # a full-size tree at the benchmark's leaf cutoff, checked on stratified outputs the oracle
    # computes one by one
    cfg = W.configs.sweep(shape=shape, n=n, d=16, kernel="exp")
    t = cfg["tree"]
    F = W.normal_field(t.n, 16, seed=123)
    p = tfi.Plan.from_spec(t, cfg["delta"], cfg["kernel"], leaf_max=leaf_max, max_channels=16, **flags)
    targets, n_classes = _stratified_targets(p, t.n, seed=1, per=per, n_random=n_random)
    assert len(targets) >= min_targets
    x = torch.from_numpy(F).cuda()
    y = p.apply(x).cpu().numpy()[targets]
    gF = p.apply_backward(x).cpu().numpy()[targets]
    ref = brute.integrate(t, cfg["delta"], cfg["kernel"], F.astype(np.float64), targets=targets)
    assert _err(y, ref) <= TOL["f32"]
    assert _err(gF, ref) <= TOL["f32"]
    return p, n_classes


def test_full_size_stratified_rrt_2p20_bench_config():
    # the benchmarked configuration itself: N = 2^20, s0 = 768 (bench.py's default leaf cutoff:
    # tensor-core leaves of up to 768 vertices, FFT classes, direct tables)
    p, n_classes = _full_size_case("rrt", 1 << 20, 768, per=128, n_random=256, min_targets=512)
    assert n_classes >= 2 and p.info()["n_jobs_direct"] > 0


@pytest.mark.parametrize("shape", ["binary", "caterpillar"])
def test_full_size_stratified_other_shapes_2p18(shape):
    _full_size_case(shape, 1 << 18, 512, per=48, n_random=96, min_targets=200)


def test_full_size_stratified_rrt_2p18_tensor_core_leaves():
    # the FP32 tensor-core leaf kernel (TFI_PLAN_LEAF_TC) at the benchmark's leaf cutoff
    p, _ = _full_size_case("rrt", 1 << 18, 512, per=64, n_random=128, min_targets=256, leaf_tc=True)
    assert p.info()["device_errors"] == 0


def test_full_size_sampled_rrt_2p20_small_leaves():
    cfg = W.configs.sweep(shape="rrt", n=1 << 20, d=16, kernel="exp")
    F = W.normal_field(cfg["tree"].n, 16, seed=123)
    rng = np.random.default_rng(0)
    targets = np.sort(rng.choice(cfg["tree"].n, size=48, replace=False)).astype(np.int32)
    _, y, ref = _run(cfg["tree"], cfg["delta"], cfg["kernel"], F, leaf_max=64, targets=targets)
    assert _err(y, ref) <= TOL["f32"]


def test_deterministic_and_adjoint():
    t = _rrt(3000, 5)
    spec = W.KernelSpec.gauss(0.02)
    p = tfi.Plan.from_spec(t, 1.0, spec, leaf_max=32, max_channels=8)
    x = torch.randn(t.n, 8, device="cuda")
    z = torch.randn(t.n, 8, device="cuda")
    y1 = p.apply(x)
    y2 = p.apply(x)
    assert torch.equal(y1, y2)
    kz = p.apply_backward(z)
    lhs = float((z.double() * y1.double()).sum())
    rhs = float((kz.double() * x.double()).sum())
    assert abs(lhs - rhs) <= 1e-4 * (abs(lhs) + abs(rhs) + 1.0)
    assert torch.equal(kz, p.apply(z))


def test_autograd_function():
    t = _rrt(500, 6)
    spec = W.KernelSpec.exp(0.3)
    p = tfi.Plan.from_spec(t, 1.0, spec, leaf_max=16, max_channels=4)
    x = torch.randn(t.n, 4, device="cuda", requires_grad=True)
    g = torch.randn(t.n, 4, device="cuda")
    y = tfi.integrate(x, p)
    (y * g).sum().backward()
    ref = brute.integrate(t, 1.0, spec, g.cpu().numpy())
    assert _err(x.grad.cpu().numpy(), ref) <= TOL["f32"]


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_apply_host_many_pipelined(pinned, dtype):
    # five independent host fields (the two staging slots are each reused), pinned and pageable,
    # against the oracle on the same (dtype-rounded) inputs
    t = _rrt(3000, 8)
    spec = W.KernelSpec.rational(0.05, e=1.0, p=2.0)
    d = 8
    p = tfi.Plan.from_spec(t, 1.0, spec, leaf_max=64, max_channels=d)
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    code = tfi.DTYPE_F32 if dtype == "f32" else tfi.DTYPE_BF16
    ins = [torch.from_numpy(W.normal_field(t.n, d, seed=40 + i)).to(tdt) for i in range(5)]
    outs = [torch.full_like(x, float("nan")) for x in ins]
    if pinned:
        ins = [x.pin_memory() for x in ins]
        outs = [y.pin_memory() for y in outs]
    p.apply_host_many([x.data_ptr() for x in ins], [y.data_ptr() for y in outs], d, code)
    for x, y in zip(ins, outs):
        ref = brute.integrate(t, 1.0, spec, x.double().numpy())
        assert _err(y.double().numpy(), ref) <= TOL[dtype]


def test_apply_host_matches_device():
    t = _rrt(2500, 8)
    p = tfi.Plan.from_spec(t, 1.0, W.KernelSpec.exp(0.2), leaf_max=64, max_channels=16)
    F = W.normal_field(t.n, 16, seed=3)
    yd = p.apply(torch.from_numpy(F).cuda()).cpu().numpy()
    yh = p.apply_host(F)
    assert np.array_equal(yd, yh)


@pytest.mark.parametrize("n,edges", [(1, []), (2, [(0, 1)]), (5, [(0, 1), (3, 4)]), (7, [])])
def test_degenerate_trees(n, edges):
    u = [a for a, _ in edges]
    v = [b for _, b in edges]
    w = [1.5] * len(edges)
    t = W.trees.Tree(n, np.array(u, np.int32), np.array(v, np.int32), np.array(w))
    F = W.normal_field(n, 5, seed=1)
    for s0 in (1, 4):
        _, y, ref = _run(t, 0.5, W.KernelSpec.exp(0.7), F, leaf_max=s0)
        assert _err(y, ref) <= TOL["f32"]


def test_largest_leaf_and_odd_channels():
    t = _rrt(3000, 9, 1, 3)
    F = W.normal_field(t.n, 7, seed=2)
    _, y, ref = _run(t, 1.0, W.KernelSpec.rational(0.5, e=2.0), F, leaf_max=1024)
    assert _err(y, ref) <= TOL["f32"]


def test_sampled_table_kernel():
    t = _rrt(1500, 10)
    tab = 1.0 / (1.0 + np.arange(400) ** 1.5 / 10.0)
    F = W.normal_field(t.n, 4, seed=4)
    _, y, ref = _run(t, 1.0, W.KernelSpec.samples(tab), F, leaf_max=32)
    assert _err(y, ref) <= TOL["f32"]


def test_stage_profile_and_model():
    t = _rrt(20000, 12)
    p = tfi.Plan.from_spec(t, 1.0, W.KernelSpec.exp(0.1), leaf_max=64, max_channels=16)
    x = torch.randn(t.n, 16, device="cuda")
    p.profile(True)
    p.apply(x)
    prof = p.profile_read()
    p.profile(False)
    assert prof["gather"][1] == 1 and prof["gather"][0] > 0
    model = p.stage_model(16)
    assert model["bucket"][0] > 0 and model["leaf"][1] > 0


@pytest.mark.parametrize("make,delta,policy", [
    (lambda: W.configs.sweep("rrt", n=1 << 16, d=1)["tree"], 1 / 64, "adaptive"),
    (lambda: W.configs.sweep("binary", n=1 << 15, d=1)["tree"], 1 / 64, "adaptive"),
    (lambda: W.configs.sweep("caterpillar", n=1 << 13, d=1)["tree"], 1 / 64, "centroid"),
    (lambda: W.configs.rrt_n2000()["tree"], 1.0, "diameter"),
    (lambda: W.spider(8, 300), 1.0, "adaptive"),
    (lambda: W.path(5000), 1.0, "diameter"),
    (lambda: W.configs.uneven_batch(count=30, lo=4, hi=2000)["tree"], 1.0, "adaptive"),
])
def test_device_keys_bit_exact(make, delta, policy):
    # (a2) depths and backbone coordinates computed on the device equal the planner's
    t = make()
    p = tfi.Plan.from_spec(t, delta, W.KernelSpec.exp(0.1), policy=policy, leaf_max=16, max_channels=1)
    host = p.export("records")
    dev = p.export("device_keys")
    assert dev.shape[0] == host.shape[0]
    assert np.array_equal(dev[:, :2], host[:, :2])
    assert np.array_equal(dev[:, 2:4], host[:, 2:4])
    assert p.info()["device_keys_ms"] > 0


def test_graph_replay_matches_apply():
    cfg = W.configs.uneven_batch(count=25, lo=8, hi=3000, d=16)
    t = cfg["tree"]
    p = tfi.Plan.from_spec(t, cfg["delta"], cfg["kernel"], leaf_max=64, max_channels=16)
    F = torch.from_numpy(W.normal_field(t.n, 16, seed=1)).cuda()
    G = torch.from_numpy(W.normal_field(t.n, 16, seed=2)).cuda()
    out, gF = torch.empty_like(F), torch.empty_like(F)
    g = tfi.Graph(p, F, out, G, gF)
    for seed in (3, 4):
        F.copy_(torch.from_numpy(W.normal_field(t.n, 16, seed=seed)).cuda())
        g.launch()
        torch.cuda.synchronize()
        assert torch.equal(out, p.apply(F)) and torch.equal(gF, p.apply(G))
    ref = brute.integrate(t, cfg["delta"], cfg["kernel"], F.cpu().numpy().astype(np.float64))
    assert _err(out.cpu().numpy(), ref) <= TOL["f32"]


@pytest.mark.parametrize("d", [16, 17, 33, 64])
def test_misaligned_field_pointers_match_aligned(d):
    # F and out 4 bytes off a 16-byte boundary: every kernel takes its scalar-load path (bin sums,
    # tensor-core leaves and tables, gather) and must give the aligned result bit for bit
    cfg = W.configs.sweep(shape="rrt", n=4096, d=d, kernel="exp")
    t = cfg["tree"]
    p = tfi.Plan.from_spec(t, cfg["delta"], cfg["kernel"], leaf_max=512, max_channels=d)
    F = torch.from_numpy(W.normal_field(t.n, d, seed=7)).cuda()
    buf = torch.zeros(t.n * d + 1, dtype=torch.float32, device="cuda")
    Fm = buf[1:].view(t.n, d)
    Fm.copy_(F)
    obuf = torch.zeros(t.n * d + 1, dtype=torch.float32, device="cuda")
    outm = obuf[1:].view(t.n, d)
    assert Fm.data_ptr() % 16 == 4 and outm.data_ptr() % 16 == 4
    y = p.apply(F)
    p.apply(Fm, outm)
    torch.cuda.synchronize()
    assert torch.equal(y, outm)


def test_apply_rejects_bad_arguments():
    """Host-side validation of tfi_apply on a device plan: every bad argument returns
    TFI_ERR_ARG (1) before anything is launched, and the plan stays usable."""
    t = _rrt(600, 11)
    p = tfi.Plan.from_spec(t, 1.0, W.KernelSpec.exp(0.3), leaf_max=64, max_channels=8)
    F = torch.from_numpy(W.normal_field(t.n, 8, seed=5)).cuda()
    out = torch.empty_like(F)
    fn = tfi.lib().tfi_apply
    ptr = lambda x: ctypes.c_void_p(x.data_ptr())
    for d, dtype, a, b in [(0, 0, F, out), (9, 0, F, out), (-1, 0, F, out), (8, 7, F, out), (8, 0, F, F)]:
        assert fn(p._h, ptr(a), ptr(b), d, dtype, None) == 1, (d, dtype)
    assert fn(p._h, None, ptr(out), 8, 0, None) == 1
    assert fn(p._h, ptr(F), None, 8, 0, None) == 1
    ref = brute.integrate(t, 1.0, W.KernelSpec.exp(0.3), F.cpu().numpy().astype(np.float64))
    assert _err(p.apply(F).cpu().numpy(), ref) <= TOL["f32"]
    assert p.info()["device_errors"] == 0
