"""FP64 evaluation of kernel specs on the distance grid (oracle side).

The paper samples the kernel at quantised distances: after quantisation the
kernel argument is delta * dhat with dhat an integer (Appendix "Distance
quantization for FFT-Based Integrators"). Test infrastructure only.
"""
from __future__ import annotations

import numpy as np


def f_of_x(spec, x: np.ndarray) -> np.ndarray:
    """f(x) in FP64 for a non-table spec; x in original distance units."""
    x = np.asarray(x, dtype=np.float64)
    p = [float(t) for t in spec.params]
    if spec.kind == "expsum":
        out = np.zeros_like(x)
        for a, b in zip(p[0::2], p[1::2]):
            out += a * np.exp(-b * x)
        return out
    if spec.kind == "gauss":
        a, c = p
        return a * np.exp(-c * x * x)
    if spec.kind == "rational":
        a, c, e, pw = p
        return a / np.power(1.0 + c * np.power(x, e), pw)
    if spec.kind == "powexp":
        a, pw, b = p
        return a * np.power(x, pw) * np.exp(-b * x)
    raise ValueError(spec.kind)


def grid_table(spec, delta: float, kmax: int) -> np.ndarray:
    """[f(k * delta) for k = 0..kmax] in FP64."""
    if spec.kind == "table":
        t = np.asarray(spec.table, dtype=np.float64)
        if t.shape[0] < kmax + 1:
            raise ValueError("kernel table shorter than the largest grid distance")
        return t[: kmax + 1].copy()
    return f_of_x(spec, np.arange(kmax + 1, dtype=np.float64) * delta)


def grid_param_derivs(spec, delta: float, kmax: int) -> np.ndarray:
    """d f(k delta) / d theta for an expsum spec, shape (len(params), kmax+1),
    rows ordered like spec.params = [a_1, b_1, a_2, b_2, ...]."""
    assert spec.kind == "expsum"
    x = np.arange(kmax + 1, dtype=np.float64) * delta
    p = [float(t) for t in spec.params]
    rows = []
    for a, b in zip(p[0::2], p[1::2]):
        e = np.exp(-b * x)
        rows.append(e)              # d/da
        rows.append(-a * x * e)     # d/db
    return np.stack(rows)


def quantise(w: np.ndarray, delta: float) -> np.ndarray:
    """q_e = max(1, round(w_e / delta)), round half to even (Appendix
    "Distance quantization", definition of q_e)."""
    return np.maximum(1, np.rint(np.asarray(w, dtype=np.float64) / delta)).astype(np.int64)
