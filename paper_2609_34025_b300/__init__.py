"""StAd-TFI (structure-adaptive tree field integration) on one B300.

A thin Python binding over ``libtfi.so`` (C ABI in ``include/tfi.h``): it
marshals arguments only. Every step of the apply runs in the library's CUDA
kernels; there is no CPU fallback, and importing the binding fails loudly when
the library has not been built.

    plan = Plan(n, u, v, w, delta=1/64, kernel=("expsum", [1.0, 0.1]), leaf_max=64, max_channels=16)
    out = plan.apply(F)                 # F: CUDA tensor (n, d), float32 or bfloat16
    y = integrate(F, plan)              # autograd: backward is the same symmetric operator
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtfi.so")

TFI_OK = 0
_STATUS = {0: "OK", 1: "ARG", 2: "NOT_TREE", 3: "WEIGHT", 4: "GRID_OVERFLOW", 5: "OOM", 6: "CUDA", 7: "TIMEOUT",
           8: "UNSUPPORTED", 9: "NO_DEVICE"}
KERNEL_KINDS = {"table": 0, "expsum": 1, "gauss": 2, "rational": 3, "powexp": 4}
POLICIES = {"adaptive": 0, "diameter": 1, "centroid": 2}
DTYPE_F32, DTYPE_BF16 = 0, 1
EXPORTS = {"calls": (0, 7), "backbone": (1, 1), "records": (2, 5), "leaves": (3, 3), "device_keys": (4, 4),
           "leaf_packs": (5, 4), "gather_order": (6, 1), "jobs": (7, 7), "leaf_ctas": (8, 4)}


class TfiError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"tfi error {_STATUS.get(code, code)}: {msg}")
        self.code = code
        self.name = _STATUS.get(code, str(code))


class _Tree(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_edges", ctypes.c_int32), ("u", ctypes.c_void_p),
                ("v", ctypes.c_void_p), ("w", ctypes.c_void_p)]


class _Kernel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n_params", ctypes.c_int32), ("params", ctypes.c_void_p),
                ("table_len", ctypes.c_int64), ("table", ctypes.c_void_p)]


class _Options(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("policy", ctypes.c_int32), ("leaf_max", ctypes.c_int32),
                ("max_channels", ctypes.c_int32), ("flags", ctypes.c_int32), ("fft_cta_points", ctypes.c_int32)]


class _Info(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "n", "n_calls", "n_leaves", "n_levels", "n_records", "n_keys", "n_jobs_fft", "n_jobs_direct",
        "n_centroid", "sum_table", "sum_fft_points", "sum_leaf_pairs", "ftab_len", "device_bytes")] + [
        ("plan_seconds", ctypes.c_double), ("device_keys_ms", ctypes.c_double), ("n_jobs_sweep", ctypes.c_int64),
        ("hist_len", ctypes.c_int64), ("n_jobs_hankel", ctypes.c_int64), ("device_errors", ctypes.c_int64),
        ("n_jobs_fft_big", ctypes.c_int64), ("sum_fft_big_points", ctypes.c_int64), ("trunc_len", ctypes.c_int64),
        ("n_zero_bins", ctypes.c_int64)]


EXPORTED_SYMBOLS = ("tfi_plan", "tfi_apply", "tfi_apply_backward", "tfi_apply_host", "tfi_destroy",
                    "tfi_plan_get_info", "tfi_plan_export", "tfi_profile_enable", "tfi_profile_read",
                    "tfi_stage_model", "tfi_apply_static", "tfi_dense_apply", "tfi_graph_create", "tfi_graph_launch",
                    "tfi_graph_destroy", "tfi_sinkhorn", "tfi_kernel_grad", "tfi_set_kernel", "tfi_selftest_wait",
                    "tfi_autotune", "tfi_apply_host_many", "tfi_last_error")
STAGES = ("leaf", "bucket", "fft", "direct", "gather", "sweep", "hankel")
HANKEL_MODES = {None: 0, False: 0, "auto": 4, "all": 8}
SWEEP_MODES = {None: 0, False: 0, True: 2, "all": 2, "auto": 32}

_lib = None


def lib():
    """The loaded libtfi (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2609_34025_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.tfi_plan.argtypes = [ctypes.POINTER(_Tree), ctypes.POINTER(_Kernel), ctypes.POINTER(_Options),
                               ctypes.POINTER(vp)]
        L.tfi_apply.argtypes = [vp, vp, vp, i32, i32, vp]
        L.tfi_apply_backward.argtypes = [vp, vp, vp, i32, i32, vp]
        L.tfi_apply_host.argtypes = [vp, vp, vp, i32, i32, vp]
        L.tfi_dense_apply.argtypes = [vp, vp, vp, i32, i32, vp]
        L.tfi_graph_create.argtypes = [vp, vp, vp, vp, vp, i32, i32, vp, ctypes.POINTER(vp)]
        L.tfi_graph_launch.argtypes = [vp, vp]
        L.tfi_graph_destroy.argtypes = [vp]
        L.tfi_sinkhorn.argtypes = [vp, vp, vp, vp, vp, i32, i32, ctypes.c_double, vp]
        L.tfi_kernel_grad.argtypes = [vp, vp, vp, i32, i32, vp, i64, vp, vp]
        L.tfi_set_kernel.argtypes = [vp, ctypes.POINTER(_Kernel)]
        L.tfi_destroy.argtypes = [vp]
        L.tfi_plan_get_info.argtypes = [vp, ctypes.POINTER(_Info)]
        L.tfi_plan_export.argtypes = [vp, i32, vp, i64, ctypes.POINTER(i64)]
        L.tfi_profile_enable.argtypes = [vp, i32]
        L.tfi_profile_read.argtypes = [vp, vp, vp]
        L.tfi_stage_model.argtypes = [vp, i32, i32, vp, vp]
        L.tfi_last_error.restype = ctypes.c_char_p
        for name in EXPORTED_SYMBOLS[:-1]:
            getattr(L, name).restype = i32
        _lib = L
    return _lib


def _check(code: int):
    if code != TFI_OK:
        raise TfiError(code, lib().tfi_last_error().decode())


def _stream_handle(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype_code(t):
    import torch

    if t.dtype == torch.float32:
        return DTYPE_F32
    if t.dtype == torch.bfloat16:
        return DTYPE_BF16
    raise TypeError(f"unsupported dtype {t.dtype}")


class Plan:
    """A planned tree (or forest): the decomposition, f samples and spectra on the device."""

    def __init__(self, n, u, v, w, delta=1.0, kernel=("expsum", [1.0, 1.0]), table=None, policy="adaptive",
                 leaf_max=64, max_channels=16, host_only=False, sweep=False, hankel=None, leaf_alu=False,
                 fft_big_all=False, fft_cta_points=0, truncate=True, direct_all=False, leaf_tc=False,
                 tables_alu=False):
        u = np.ascontiguousarray(u, dtype=np.int32)
        v = np.ascontiguousarray(v, dtype=np.int32)
        w = np.ascontiguousarray(w, dtype=np.float64)
        kind, params = kernel
        params = np.ascontiguousarray(params, dtype=np.float64)
        tab = None if table is None else np.ascontiguousarray(table, dtype=np.float64)
        tree = _Tree(int(n), int(u.shape[0]), u.ctypes.data, v.ctypes.data, w.ctypes.data)
        ker = _Kernel(KERNEL_KINDS[kind], int(params.shape[0]), params.ctypes.data if params.size else None,
                      0 if tab is None else int(tab.shape[0]), None if tab is None else tab.ctypes.data)
        opt = _Options(float(delta), POLICIES[policy], int(leaf_max), int(max_channels),
                       (1 if host_only else 0) | SWEEP_MODES[sweep] | HANKEL_MODES[hankel] | (16 if leaf_alu else 0)
                       | (64 if fft_big_all else 0) | (0 if truncate else 128) | (256 if direct_all else 0)
                       | (512 if leaf_tc else 0) | (1024 if tables_alu else 0),
                       int(fft_cta_points))
        h = ctypes.c_void_p()
        _check(lib().tfi_plan(ctypes.byref(tree), ctypes.byref(ker), ctypes.byref(opt), ctypes.byref(h)))
        self._h = h
        self.n = int(n)
        self.max_channels = int(max_channels)
        self.host_only = host_only
        self.kernel_kind = KERNEL_KINDS[kind]
        self.n_params = 0 if kind == "table" else int(params.shape[0])

    @classmethod
    def autotune(cls, tree, delta, spec, d, dtype="f32", leaf_candidates=None, sample_trees=0, reps=5,
                 policy="adaptive", max_channels=None, **flags):
        """Plan with the leaf cutoff and FFT tile that measure fastest for d channels (tfi_autotune).
        Returns (plan, {"leaf_max", "fft_cta_points", "ms_per_apply"})."""
        u = np.ascontiguousarray(tree.u, dtype=np.int32)
        v = np.ascontiguousarray(tree.v, dtype=np.int32)
        w = np.ascontiguousarray(tree.w, dtype=np.float64)
        params = np.ascontiguousarray(list(spec.params), dtype=np.float64)
        tab = None if getattr(spec, "table", None) is None else np.ascontiguousarray(spec.table, dtype=np.float64)
        tr = _Tree(int(tree.n), int(u.shape[0]), u.ctypes.data, v.ctypes.data, w.ctypes.data)
        ker = _Kernel(KERNEL_KINDS[spec.kind], int(params.shape[0]), params.ctypes.data if params.size else None,
                      0 if tab is None else int(tab.shape[0]), None if tab is None else tab.ctypes.data)
        mc = int(max_channels or d)
        fl = SWEEP_MODES[flags.get("sweep", False)] | HANKEL_MODES[flags.get("hankel", None)] | \
            (16 if flags.get("leaf_alu") else 0) | (64 if flags.get("fft_big_all") else 0) | \
            (512 if flags.get("leaf_tc") else 0) | (1024 if flags.get("tables_alu") else 0)
        opt = _Options(float(delta), POLICIES[policy], 64, mc, fl, 0)
        cand = None if leaf_candidates is None else np.ascontiguousarray(leaf_candidates, dtype=np.int32)
        tuned = _Options()
        ms = ctypes.c_double()
        h = ctypes.c_void_p()
        dt = DTYPE_F32 if dtype in ("f32", DTYPE_F32) else DTYPE_BF16
        _check(lib().tfi_autotune(ctypes.byref(tr), ctypes.byref(ker), ctypes.byref(opt), int(d), dt,
                                  None if cand is None else cand.ctypes.data, 0 if cand is None else int(cand.shape[0]),
                                  int(sample_trees), int(reps), ctypes.byref(tuned), ctypes.byref(ms), ctypes.byref(h)))
        plan = cls.__new__(cls)
        plan._h = h
        plan.n = int(tree.n)
        plan.max_channels = mc
        plan.host_only = False
        plan.kernel_kind = KERNEL_KINDS[spec.kind]
        plan.n_params = 0 if spec.kind == "table" else int(params.shape[0])
        return plan, {"leaf_max": int(tuned.leaf_max), "fft_cta_points": int(tuned.fft_cta_points),
                      "ms_per_apply": float(ms.value)}

    @classmethod
    def from_spec(cls, tree, delta, spec, **kw):
        """Build from any tree with (n, u, v, w) and a kernel spec with (kind, params, table)."""
        return cls(tree.n, tree.u, tree.v, tree.w, delta=delta, kernel=(spec.kind, list(spec.params)),
                   table=getattr(spec, "table", None), **kw)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().tfi_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _apply(self, fn, F, out, stream):
        import torch

        if not F.is_cuda or F.dim() != 2 or F.shape[0] != self.n or not F.is_contiguous():
            raise ValueError("F must be a contiguous CUDA tensor of shape (n, d)")
        if out is None:
            out = torch.empty_like(F)
        if out.shape != F.shape or out.dtype != F.dtype or not out.is_contiguous():
            raise ValueError("out must match F")
        _check(fn(self._h, ctypes.c_void_p(F.data_ptr()), ctypes.c_void_p(out.data_ptr()), int(F.shape[1]),
                  _dtype_code(F), _stream_handle(stream)))
        return out

    def apply(self, F, out=None, stream=None):
        """out = K F on the device (stream-ordered)."""
        return self._apply(lib().tfi_apply, F, out, stream)

    def dense_apply(self, F, out=None, stream=None):
        """out = K F by dense tensor-core evaluation per tree (synchronises)."""
        return self._apply(lib().tfi_dense_apply, F, out, stream)

    def sinkhorn(self, a, b, iters=200, delta_reg=1e-30, stream=None):
        """Sinkhorn scalings (u, v) for marginal pairs a, b (CUDA float32, n x d)."""
        import torch

        for t in (a, b):
            if not t.is_cuda or t.dtype != torch.float32 or t.shape[0] != self.n or not t.is_contiguous():
                raise ValueError("marginals must be contiguous CUDA float32 tensors of shape (n, d)")
        u, v = torch.empty_like(a), torch.empty_like(a)
        _check(lib().tfi_sinkhorn(self._h, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                  ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(v.data_ptr()), int(a.shape[1]),
                                  int(iters), float(delta_reg), _stream_handle(stream)))
        return u, v

    def kernel_grad(self, grad_out, F, stream=None, device_dtheta=False):
        """(C, dtheta): C[k] = dL/df(k delta) (CUDA float64) and dL/dtheta for grad_out = dL/dout;
        dtheta is a numpy array (the call synchronises), or with device_dtheta a CUDA float64 tensor
        written on the stream (no synchronisation)."""
        import torch

        for t in (grad_out, F):
            if not t.is_cuda or t.dim() != 2 or t.shape[0] != self.n or not t.is_contiguous():
                raise ValueError("grad_out and F must be contiguous CUDA tensors of shape (n, d)")
        if getattr(self, "_hist_len", None) is None:
            self._hist_len = self.info()["hist_len"]
        L = self._hist_len
        C = torch.empty(L, dtype=torch.float64, device=grad_out.device)
        if device_dtheta:
            th = torch.zeros(max(1, self.n_params), dtype=torch.float64, device=grad_out.device)
            th_ptr = ctypes.c_void_p(th.data_ptr()) if self.n_params else None
        else:
            th = np.zeros(max(1, self.n_params), dtype=np.float64)
            th_ptr = th.ctypes.data if self.n_params else None
        _check(lib().tfi_kernel_grad(self._h, ctypes.c_void_p(grad_out.data_ptr()), ctypes.c_void_p(F.data_ptr()),
                                     int(F.shape[1]), _dtype_code(F), ctypes.c_void_p(C.data_ptr()), L,
                                     th_ptr, _stream_handle(stream)))
        if stream is not None:
            # written on `stream`: keep the caching allocator from reusing them before it is done
            C.record_stream(stream)
            if device_dtheta:
                th.record_stream(stream)
        return C, th[: self.n_params]

    def set_kernel(self, params=None, table=None):
        """Replace f's parameters (same kind and count) or its sampled table, without replanning."""
        params = np.ascontiguousarray(params if params is not None else [], dtype=np.float64)
        tab = None if table is None else np.ascontiguousarray(table, dtype=np.float64)
        ker = _Kernel(self.kernel_kind, int(params.shape[0]), params.ctypes.data if params.size else None,
                      0 if tab is None else int(tab.shape[0]), None if tab is None else tab.ctypes.data)
        _check(lib().tfi_set_kernel(self._h, ctypes.byref(ker)))
        self.n_params = int(params.shape[0]) if tab is None else 0

    def apply_backward(self, grad_out, out=None, stream=None):
        """grad_F = K^T grad_out (= K grad_out: the operator is symmetric)."""
        return self._apply(lib().tfi_apply_backward, grad_out, out, stream)

    def apply_host(self, F: np.ndarray, out: np.ndarray | None = None, stream=None) -> np.ndarray:
        """Host arrays in and out: copies, apply, copies back, synchronised."""
        if F.dtype != np.float32 or F.ndim != 2 or F.shape[0] != self.n:
            raise ValueError("F must be float32 of shape (n, d)")
        F = np.ascontiguousarray(F)
        if out is None:
            out = np.empty_like(F)
        _check(lib().tfi_apply_host(self._h, ctypes.c_void_p(F.ctypes.data), ctypes.c_void_p(out.ctypes.data),
                                    int(F.shape[1]), DTYPE_F32, _stream_handle(stream)))
        return out

    def apply_host_ptr(self, f_ptr: int, out_ptr: int, d: int, dtype: int = DTYPE_F32, stream=None):
        """Host pointers (e.g. pinned torch tensors) in and out, synchronised."""
        _check(lib().tfi_apply_host(self._h, ctypes.c_void_p(f_ptr), ctypes.c_void_p(out_ptr), int(d), int(dtype),
                                    _stream_handle(stream)))

    def apply_host_many(self, f_ptrs, out_ptrs, d: int, dtype: int = DTYPE_F32, stream=None):
        """Host fields in and out (e.g. pinned torch tensors), pipelined copies and applies, synchronised."""
        n = len(f_ptrs)
        if len(out_ptrs) != n:
            raise ValueError("need one output per input")
        fa = (ctypes.c_void_p * max(1, n))(*[ctypes.c_void_p(p) for p in f_ptrs])
        oa = (ctypes.c_void_p * max(1, n))(*[ctypes.c_void_p(p) for p in out_ptrs])
        _check(lib().tfi_apply_host_many(self._h, n, fa, oa, int(d), int(dtype), _stream_handle(stream)))

    def info(self) -> dict:
        inf = _Info()
        _check(lib().tfi_plan_get_info(self._h, ctypes.byref(inf)))
        return {name: getattr(inf, name) for name, _ in _Info._fields_}

    def selftest_wait(self, arrive: bool, max_polls: int = 10_000, stream=None) -> bool:
        """Run the bounded-wait self-test (tfi_selftest_wait): True if the wait completed, False if
        it ran out of polls (TFI_ERR_TIMEOUT; the plan's device_errors then counts it)."""
        code = lib().tfi_selftest_wait(self._h, int(bool(arrive)), int(max_polls), _stream_handle(stream))
        if code == 7:  # TFI_ERR_TIMEOUT
            return False
        _check(code)
        return True

    def profile(self, enable: bool = True, serialize: bool = False):
        """Start (clearing totals) or stop per-stage CUDA-event timing; serialize runs every stage
        on the caller's stream, so each stage is timed alone."""
        _check(lib().tfi_profile_enable(self._h, (2 if serialize else 1) if enable else 0))

    def profile_read(self) -> dict:
        """{stage: (milliseconds, launches)} summed since profiling was enabled (synchronises)."""
        ms = np.zeros(len(STAGES), dtype=np.float64)
        ln = np.zeros(len(STAGES), dtype=np.int64)
        _check(lib().tfi_profile_read(self._h, ms.ctypes.data, ln.ctypes.data))
        return {k: (float(ms[i]), int(ln[i])) for i, k in enumerate(STAGES)}

    def stage_model(self, d: int, dtype: int = DTYPE_F32) -> dict:
        """{stage: (algorithmic bytes, flops)} for one apply with d channels."""
        b = np.zeros(len(STAGES), dtype=np.float64)
        f = np.zeros(len(STAGES), dtype=np.float64)
        _check(lib().tfi_stage_model(self._h, int(d), int(dtype), b.ctypes.data, f.ctypes.data))
        return {k: (float(b[i]), float(f[i])) for i, k in enumerate(STAGES)}

    def export(self, what: str) -> np.ndarray:
        """The plan's decomposition or launch layout as an int64 array (one row per item):
        "calls" (level, min vertex, |V(S)|, kind, m, H, L), "backbone" (p_1..p_m of every call),
        "records" (call, vertex, depth, coordinate, component), "leaves" (level, min vertex, size),
        "device_keys" (call, vertex, device depth, device coordinate; device plans only),
        "leaf_packs" (CTA, leaf begin, leaf end, CTA vertex capacity), "gather_order"
        (vertices in the gather's order), "jobs" (evaluator, log2 FFT points, is correction,
        bins, first member vertex, last member vertex, largest depth) and "leaf_ctas" (CTA, leaf
        begin, leaf end, CTA count of the FP32 tensor-core leaf kernel)."""
        code, width = EXPORTS[what]
        ln = ctypes.c_int64()
        _check(lib().tfi_plan_export(self._h, code, None, 0, ctypes.byref(ln)))
        buf = np.empty(ln.value, dtype=np.int64)
        _check(lib().tfi_plan_export(self._h, code, buf.ctypes.data if ln.value else None, ln.value,
                                     ctypes.byref(ln)))
        return buf.reshape(-1, width) if width > 1 else buf


class Graph:
    """A captured forward (+ optional backward) step on fixed buffers, replayed by one graph launch."""

    def __init__(self, plan: Plan, F, out, grad_out=None, grad_F=None, stream=None):
        self.plan = plan
        self.bufs = (F, out, grad_out, grad_F)  # keep the buffers alive
        h = ctypes.c_void_p()
        ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
        _check(lib().tfi_graph_create(plan._h, ptr(F), ptr(out), ptr(grad_out), ptr(grad_F), int(F.shape[1]),
                                      _dtype_code(F), _stream_handle(stream), ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        _check(lib().tfi_graph_launch(self._h, _stream_handle(stream)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().tfi_graph_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd_fn():
    import torch

    class TreeFieldIntegral(torch.autograd.Function):
        """y = K F with dL/dF = K dL/dy (K symmetric)."""

        @staticmethod
        def forward(ctx, F, plan):
            ctx.plan = plan
            return plan.apply(F.contiguous())

        @staticmethod
        def backward(ctx, g):
            return ctx.plan.apply_backward(g.contiguous()), None

    return TreeFieldIntegral


def _learnable_fn():
    import torch

    class LearnableKernelIntegral(torch.autograd.Function):
        """y = K_theta F with dL/dF = K_theta dL/dy and dL/dtheta = sum_k df(k delta)/dtheta C[k]."""

        @staticmethod
        def forward(ctx, F, theta, plan):
            plan.set_kernel(params=theta.detach().double().cpu().numpy())
            ctx.plan = plan
            ctx.save_for_backward(F)
            ctx.theta_dtype = theta.dtype
            return plan.apply(F.contiguous())

        @staticmethod
        def backward(ctx, g):
            (F,) = ctx.saved_tensors
            g = g.contiguous()
            dF = ctx.plan.apply_backward(g)
            _, dth = ctx.plan.kernel_grad(g, F.contiguous())
            return dF, torch.from_numpy(dth).to(dtype=ctx.theta_dtype), None

    return LearnableKernelIntegral


_TFI = None
_LTFI = None


def integrate_learnable(F, theta, plan: Plan):
    """Differentiable in F and in the kernel parameters theta (1-D tensor in the
    order of the plan's kernel params): sets the plan's kernel to theta, applies,
    and back-propagates through the hand-written adjoint and kernel gradient."""
    global _LTFI
    if _LTFI is None:
        _LTFI = _learnable_fn()
    return _LTFI.apply(F, theta, plan)


def integrate(F, plan: Plan):
    """Differentiable out = K F (autograd through the hand-written adjoint)."""
    global _TFI
    if _TFI is None:
        _TFI = _autograd_fn()
    return _TFI.apply(F, plan)
