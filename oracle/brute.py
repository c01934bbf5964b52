"""FP64 brute-force oracle (plain definition, Eq. "integration" / "stad-target").

Test infrastructure only: see ``oracle/__init__.py``. The arithmetic lives in
``brute.c`` (one traversal per target, FP64 sums); this module quantises the
edge lengths, evaluates f on the grid and marshals arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from .kernels import grid_table, quantise

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "brute.c")
_LIB = os.path.join(_HERE, "_brute.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile brute.c into _brute.so (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        p = ctypes.c_void_p
        lib.tfi_oracle_max_dist.restype = ctypes.c_int64
        lib.tfi_oracle_max_dist.argtypes = [ctypes.c_int32, p, p, p]
        lib.tfi_oracle_apply.restype = ctypes.c_int
        lib.tfi_oracle_apply.argtypes = [ctypes.c_int32, p, p, p, p, ctypes.c_int64, p, ctypes.c_int32,
                                         p, ctypes.c_int64, p, ctypes.c_int32]
        lib.tfi_oracle_corr_hist.restype = ctypes.c_int
        lib.tfi_oracle_corr_hist.argtypes = [ctypes.c_int32, p, p, p, p, p, ctypes.c_int32,
                                             p, ctypes.c_int64, p, ctypes.c_int64, ctypes.c_int32]
        lib.tfi_oracle_dist_rows.restype = None
        lib.tfi_oracle_dist_rows.argtypes = [ctypes.c_int32, p, p, p, p, ctypes.c_int64, p]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Adjacency:
    """CSR adjacency (neighbours sorted by id) with quantised integer lengths."""

    def __init__(self, tree, delta: float):
        n = tree.n
        q = quantise(tree.w, delta)
        a = np.concatenate([tree.u, tree.v]).astype(np.int64)
        b = np.concatenate([tree.v, tree.u]).astype(np.int64)
        ql = np.concatenate([q, q])
        order = np.lexsort((b, a))
        a, b, ql = a[order], b[order], ql[order]
        self.n = n
        self.q = q
        self.ptr = np.zeros(n + 1, dtype=np.int64)
        np.add.at(self.ptr, a + 1, 1)
        self.ptr = np.cumsum(self.ptr).astype(np.int64)
        self.adj = np.ascontiguousarray(b, dtype=np.int32)
        self.len = np.ascontiguousarray(ql, dtype=np.int64)
        self._maxd = None

    def max_dist(self) -> int:
        if self._maxd is None:
            self._maxd = int(_load().tfi_oracle_max_dist(self.n, _ptr(self.ptr), _ptr(self.adj), _ptr(self.len)))
        return self._maxd

    def dist_rows(self, sources) -> np.ndarray:
        src = np.ascontiguousarray(sources, dtype=np.int32)
        rows = np.empty((src.shape[0], self.n), dtype=np.int64)
        _load().tfi_oracle_dist_rows(self.n, _ptr(self.ptr), _ptr(self.adj), _ptr(self.len), _ptr(src),
                                     src.shape[0], _ptr(rows))
        return rows


def integrate(tree, delta: float, spec, F: np.ndarray, targets=None, threads: int = 0, adj: Adjacency | None = None):
    """out[t] = sum_v f(delta * dhat(t, v)) F[v] for t in targets (all if None).

    F: (n, d) or (n,) array (converted to FP64). Returns FP64 (len(targets), d)
    (or (n,) for a 1-D field with targets=None).
    """
    adj = adj or Adjacency(tree, delta)
    F = np.asarray(F, dtype=np.float64)
    squeeze = F.ndim == 1
    if squeeze:
        F = F[:, None]
    F = np.ascontiguousarray(F)
    n, d = F.shape
    assert n == tree.n
    tgt = np.arange(n, dtype=np.int32) if targets is None else np.ascontiguousarray(targets, dtype=np.int32)
    ftab = np.ascontiguousarray(grid_table(spec, delta, adj.max_dist()))
    out = np.empty((tgt.shape[0], d), dtype=np.float64)
    bad = _load().tfi_oracle_apply(n, _ptr(adj.ptr), _ptr(adj.adj), _ptr(adj.len), _ptr(ftab), ftab.shape[0],
                                   _ptr(F), d, _ptr(tgt), tgt.shape[0], _ptr(out), int(threads))
    if bad:
        raise RuntimeError("distance beyond kernel table")
    if squeeze and targets is None:
        return out[:, 0]
    return out


def corr_hist(tree, delta: float, G: np.ndarray, F: np.ndarray, targets=None, threads: int = 0,
              adj: Adjacency | None = None) -> np.ndarray:
    """hist[k] = sum_{u in targets} sum_{v : dhat(u,v) = k} <G[u], F[v]>, k = 0..maxdist."""
    adj = adj or Adjacency(tree, delta)
    G = np.ascontiguousarray(np.asarray(G, dtype=np.float64).reshape(tree.n, -1))
    F = np.ascontiguousarray(np.asarray(F, dtype=np.float64).reshape(tree.n, -1))
    d = F.shape[1]
    tgt = np.arange(tree.n, dtype=np.int32) if targets is None else np.ascontiguousarray(targets, dtype=np.int32)
    tlen = adj.max_dist() + 1
    hist = np.zeros(tlen, dtype=np.float64)
    bad = _load().tfi_oracle_corr_hist(tree.n, _ptr(adj.ptr), _ptr(adj.adj), _ptr(adj.len), _ptr(G), _ptr(F), d,
                                       _ptr(tgt), tgt.shape[0], _ptr(hist), tlen, int(threads))
    if bad:
        raise RuntimeError("distance beyond histogram")
    return hist


def kernel_param_grad(tree, delta: float, spec, G: np.ndarray, F: np.ndarray, threads: int = 0) -> np.ndarray:
    """dL/dtheta for an analytic kernel, given G = dL/dout: sum_k df(k delta)/dtheta * hist[k]."""
    from .kernels import grid_param_derivs

    adj = Adjacency(tree, delta)
    hist = corr_hist(tree, delta, G, F, threads=threads, adj=adj)
    der = grid_param_derivs(spec, delta, hist.shape[0] - 1)
    return der @ hist
