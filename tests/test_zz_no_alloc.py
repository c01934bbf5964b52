"""tfi_apply_static: the allocation-free apply, for callers that must not
allocate device memory while they run (hosts whose own allocator or fixed
budget owns all device memory, latency-critical loops that cannot absorb
cudaMalloc's implicit synchronisation). Through the C ABI, on two calls in a
row, it must give the same result as tfi_apply and match the FP64 oracle, and
after its first call on the device it must leave the device's free memory and
the plan's device bytes unchanged.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test. It also passes alone in a fresh process: the
first call on the device performs the one-time symbol-address lookup.
"""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle import brute

from ._lib import tfi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {tfi.DTYPE_F32: 1e-4, tfi.DTYPE_BF16: 1e-2}


def _static_fn():
    f = tfi.lib().tfi_apply_static
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
    f.restype = ctypes.c_int32
    return f


def _err(y, ref):
    y = np.asarray(y, np.float64)
    ref = np.asarray(ref, np.float64)
    return float((np.abs(y - ref).max(0) / np.maximum(np.abs(ref).max(0), 1e-300)).max())


def _call(fn, plan, x, out, d, dt):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return fn(plan._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), d, dt, stream)


_PLANS = {}


def _plan(which):
    # one plan per workload with the widest d of the tests; smaller d reuse it
    if which not in _PLANS:
        if which == "rrt_n2000":
            cfg = W.configs.rrt_n2000()
            _PLANS[which] = (cfg, tfi.Plan.from_spec(cfg["tree"], cfg["delta"], cfg["kernel"], leaf_max=64,
                                                     max_channels=64))
        else:
            # the grid-1/64 random recursive tree at N=4096: FFT correction tables, direct tables,
            # packed big leaves and small leaves
            cfg = W.configs.sweep("rrt", n=4096, d=16)
            _PLANS[which] = (cfg, tfi.Plan.from_spec(cfg["tree"], cfg["delta"], cfg["kernel"], leaf_max=256,
                                                     max_channels=64))
    return _PLANS[which]


@pytest.mark.parametrize("which", ["rrt_n2000", "rrt_n4096_grid64"])
@pytest.mark.parametrize("dt", [tfi.DTYPE_F32, tfi.DTYPE_BF16], ids=["f32", "bf16"])
@pytest.mark.parametrize("d", [1, 3, 16, 64])
def test_static_apply_matches_apply_and_oracle_on_two_calls(which, dt, d):
    cfg, plan = _plan(which)
    t = cfg["tree"]
    if which != "rrt_n2000":
        assert plan.info()["n_jobs_fft"] > 0
    tdt = torch.float32 if dt == tfi.DTYPE_F32 else torch.bfloat16
    fn = _static_fn()
    free_after_first = None
    bytes_before = plan.info()["device_bytes"]
    for seed in (123, 321):  # two calls in a row, different inputs
        x = torch.from_numpy(W.normal_field(t.n, d, seed=seed)).cuda().to(tdt)
        ref = plan.apply(x).double().cpu().numpy()
        out = torch.full_like(x, float("nan"))
        rc = _call(fn, plan, x, out, d, dt)
        assert rc == 0, tfi.lib().tfi_last_error().decode()
        torch.cuda.synchronize()
        if free_after_first is None:
            free_after_first = torch.cuda.mem_get_info()[0]
        else:
            assert torch.cuda.mem_get_info()[0] == free_after_first
        y = out.double().cpu().numpy()
        assert np.isfinite(y).all()
        want = brute.integrate(t, cfg["delta"], cfg["kernel"], x.double().cpu().numpy())
        assert _err(y, want) <= TOL[dt]
        assert _err(y, ref) <= TOL[dt]
    assert plan.info()["device_bytes"] == bytes_before


def test_static_apply_rejects_oversized_plans():
    t = W.random_recursive(200_000, np.random.default_rng(0))
    plan = tfi.Plan.from_spec(t, 1.0, W.KernelSpec.exp(0.1), leaf_max=16, max_channels=16)
    x = torch.zeros(t.n, 16, device="cuda")
    out = torch.empty_like(x)
    assert _call(_static_fn(), plan, x, out, 16, tfi.DTYPE_F32) == 1  # TFI_ERR_ARG
    assert "static workspace" in tfi.lib().tfi_last_error().decode()


@pytest.mark.parametrize("mode", ["sweep", "hankel"])
def test_static_apply_rejects_sweep_and_hankel_plans(mode):
    cfg = W.configs.attention(heads=1)
    h = cfg["heads"][0]
    kw = dict(sweep=True) if mode == "sweep" else dict(hankel="all")
    plan = tfi.Plan.from_spec(h["tree"], 1.0, h["kernel"], leaf_max=1, max_channels=16, **kw)
    info = plan.info()
    assert (info["n_jobs_sweep"] if mode == "sweep" else info["n_jobs_hankel"]) > 0
    x = torch.zeros(h["tree"].n, 16, device="cuda")
    out = torch.empty_like(x)
    assert _call(_static_fn(), plan, x, out, 16, tfi.DTYPE_F32) == 8  # TFI_ERR_UNSUPPORTED
