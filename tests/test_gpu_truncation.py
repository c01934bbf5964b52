"""Support truncation (TFI_PLAN_NO_TRUNCATE turns it off): when every FP32 kernel
sample from some distance T on is zero, bins at depth >= T are left out of their
tables with zero values. Through the C ABI against the FP64 oracle and against
the same plan without truncation; the kernel gradient still counts every pair;
a new kernel with a longer support is refused."""
import numpy as np
import pytest

import workloads as W
from oracle import brute

from ._lib import tfi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _err(y, ref):
    y = np.asarray(y, dtype=np.float64).reshape(ref.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return float((np.abs(y - ref).max(0) / np.maximum(np.abs(ref).max(0), 1e-300)).max())


def _run(p, F):
    y = p.apply(torch.from_numpy(F).cuda())
    torch.cuda.synchronize()
    return y.double().cpu().numpy()


@pytest.mark.parametrize("shape,n,kernel", [("caterpillar", 1 << 14, "exp"), ("caterpillar", 1 << 14, "gauss"),
                                            ("caterpillar", 1 << 12, "gauss")])
@pytest.mark.parametrize("d", [3, 16])
def test_truncated_plans_match_oracle_and_untruncated(shape, n, kernel, d):
    cfg = W.configs.sweep(shape=shape, n=n, d=d, kernel=kernel)
    t = cfg["tree"]
    p = tfi.Plan.from_spec(t, cfg["delta"], cfg["kernel"], leaf_max=64, max_channels=d)
    q = tfi.Plan.from_spec(t, cfg["delta"], cfg["kernel"], leaf_max=64, max_channels=d, truncate=False)
    info = p.info()
    assert info["trunc_len"] >= 0 and info["n_zero_bins"] > 0 and q.info()["trunc_len"] == -1
    F = W.normal_field(t.n, d, seed=123)
    y = _run(p, F)
    assert _err(y, brute.integrate(t, cfg["delta"], cfg["kernel"], F.astype(np.float64))) <= 1e-4
    assert _err(y, _run(q, F)) <= 1e-5


def test_truncated_torus_sinkhorn_operator():
    cfg = W.configs.torus_sinkhorn(n=4000, pairs=8)
    t = cfg["tree"]
    p = tfi.Plan.from_spec(t, cfg["delta"], cfg["kernel"], leaf_max=64, max_channels=8)
    assert p.info()["trunc_len"] >= 0
    a, _ = W.dirichlet_pairs(t.n, 8, seed=1)
    assert _err(_run(p, a.astype(np.float32)), brute.integrate(t, cfg["delta"], cfg["kernel"], a.astype(np.float64))) <= 1e-4


def test_set_kernel_on_a_truncated_plan():
    t = W.configs.rrt_n2000()["tree"]
    spec = W.KernelSpec.gauss(0.3)
    p = tfi.Plan.from_spec(t, 1.0, spec, leaf_max=16, max_channels=4)
    assert p.info()["trunc_len"] >= 0
    F = W.normal_field(t.n, 4, seed=9)
    # a faster decay (shorter support) is accepted and exact
    p.set_kernel(params=[1.0, 0.6])
    assert _err(_run(p, F), brute.integrate(t, 1.0, W.KernelSpec("gauss", [1.0, 0.6]), F.astype(np.float64))) <= 1e-4
    # a slower decay would need the cut bins: refused, plan unchanged
    with pytest.raises(tfi.TfiError) as e:
        p.set_kernel(params=[1.0, 0.01])
    assert e.value.name == "UNSUPPORTED"
    assert _err(_run(p, F), brute.integrate(t, 1.0, W.KernelSpec("gauss", [1.0, 0.6]), F.astype(np.float64))) <= 1e-4
    # without truncation any kernel of the kind is accepted
    q = tfi.Plan.from_spec(t, 1.0, spec, leaf_max=16, max_channels=4, truncate=False)
    q.set_kernel(params=[1.0, 0.01])
    assert _err(_run(q, F), brute.integrate(t, 1.0, W.KernelSpec("gauss", [1.0, 0.01]), F.astype(np.float64))) <= 1e-4


def test_kernel_grad_counts_every_pair_on_a_truncated_plan():
    cfg = W.configs.rrt_n2000()
    t = cfg["tree"]
    spec = W.KernelSpec.gauss(0.3)
    p = tfi.Plan.from_spec(t, 1.0, spec, leaf_max=16, max_channels=8)
    assert p.info()["n_zero_bins"] > 0
    G = torch.from_numpy(W.normal_field(t.n, 8, seed=31)).cuda()
    F = torch.from_numpy(W.normal_field(t.n, 8, seed=32)).cuda()
    C, dth = p.kernel_grad(G, F)
    Gn, Fn = G.double().cpu().numpy(), F.double().cpu().numpy()
    ref = brute.corr_hist(t, 1.0, Gn, Fn)
    c = C.cpu().numpy()
    ref = np.concatenate([ref, np.zeros(len(c) - len(ref))])
    assert float(np.abs(c - ref).max() / np.abs(ref).max()) <= 1e-4
    dref = brute.kernel_param_grad(t, 1.0, spec, Gn, Fn)
    assert float(np.abs(np.asarray(dth) - dref).max() / np.abs(dref).max()) <= 1e-4


def test_static_apply_on_a_truncated_plan():
    import ctypes
    cfg = W.configs.sweep(shape="caterpillar", n=4096, d=16, kernel="gauss")
    t = cfg["tree"]
    p = tfi.Plan.from_spec(t, cfg["delta"], cfg["kernel"], leaf_max=64, max_channels=16)
    assert p.info()["n_zero_bins"] > 0
    f = tfi.lib().tfi_apply_static
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
    f.restype = ctypes.c_int32
    x = torch.from_numpy(W.normal_field(t.n, 16, seed=5)).cuda()
    out = torch.full_like(x, float("nan"))
    assert f(p._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), 16, tfi.DTYPE_F32,
             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    torch.cuda.synchronize()
    ref = brute.integrate(t, cfg["delta"], cfg["kernel"], x.double().cpu().numpy())
    assert _err(out.double().cpu().numpy(), ref) <= 1e-4
