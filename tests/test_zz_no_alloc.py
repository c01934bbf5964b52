"""tfi_apply_static: the allocation-free apply, for callers that must not
allocate device memory while they run (hosts whose own allocator or fixed
budget owns all device memory, latency-critical loops that cannot absorb
cudaMalloc's implicit synchronisation). It must give the same result as
tfi_apply on consecutive calls, through the C ABI.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test. It also passes alone in a fresh process: the
first call on the device performs the one-time symbol-address lookup.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

from ._lib import tfi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _static_fn():
    f = tfi.lib().tfi_apply_static
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
    f.restype = ctypes.c_int32
    return f


def _err(y, ref):
    y = y.double().cpu().numpy()
    ref = ref.double().cpu().numpy()
    return float((np.abs(y - ref).max(0) / np.maximum(np.abs(ref).max(0), 1e-300)).max())


def test_static_apply_matches_apply_on_two_calls():
    cfg = W.configs.rrt_n2000()
    t, d = cfg["tree"], cfg["d"]
    plan = tfi.Plan.from_spec(t, cfg["delta"], cfg["kernel"], leaf_max=64, max_channels=d)
    fn = _static_fn()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed in (123, 321):  # two calls in a row, different inputs
        x = torch.from_numpy(W.normal_field(t.n, d, seed=seed)).cuda()
        ref = plan.apply(x)
        out = torch.full_like(x, float("nan"))
        rc = fn(plan._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), d, tfi.DTYPE_F32, stream)
        assert rc == 0, tfi.lib().tfi_last_error().decode()
        torch.cuda.synchronize()
        assert _err(out, ref) <= 1e-4


def test_static_apply_rejects_oversized_plans():
    t = W.random_recursive(200_000, np.random.default_rng(0))
    plan = tfi.Plan.from_spec(t, 1.0, W.KernelSpec.exp(0.1), leaf_max=16, max_channels=16)
    x = torch.zeros(t.n, 16, device="cuda")
    out = torch.empty_like(x)
    rc = _static_fn()(plan._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), 16, tfi.DTYPE_F32,
                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 1  # TFI_ERR_ARG
    assert "static workspace" in tfi.lib().tfi_last_error().decode()
