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
    """d f(k delta) / d theta, shape (len(params), kmax+1), rows in the order
    of spec.params, for every analytic kind. Derivatives of the closed forms:
      expsum   a_i e^{-b_i x}:   e^{-b_i x},  -a_i x e^{-b_i x}
      gauss    a e^{-c x^2}:     e^{-c x^2},  -a x^2 e^{-c x^2}
      rational a u^{-p}, u = 1 + c x^e:
               u^{-p},  -a p x^e u^{-p-1},  -a p c x^e ln(x) u^{-p-1},  -a ln(u) u^{-p}
      powexp   a x^p e^{-b x}:   x^p e^{-b x},  a x^p ln(x) e^{-b x},  -a x^{p+1} e^{-b x}
    At x = 0 the terms x^s ln(x) (s > 0) are taken at their limit 0."""
    x = np.arange(kmax + 1, dtype=np.float64) * delta
    p = [float(t) for t in spec.params]
    pos = x > 0
    logx = np.where(pos, np.log(np.where(pos, x, 1.0)), 0.0)
    if spec.kind == "expsum":
        rows = []
        for a, b in zip(p[0::2], p[1::2]):
            e = np.exp(-b * x)
            rows += [e, -a * x * e]
        return np.stack(rows)
    if spec.kind == "gauss":
        a, c = p
        e = np.exp(-c * x * x)
        return np.stack([e, -a * x * x * e])
    if spec.kind == "rational":
        a, c, ex, pw = p
        xe = np.where(pos, np.power(np.where(pos, x, 1.0), ex), 0.0)
        u = 1.0 + c * xe
        t = np.power(u, -pw)
        return np.stack([t, -a * pw * xe * t / u, -a * pw * c * xe * logx * t / u, -a * np.log(u) * t])
    if spec.kind == "powexp":
        a, pw, b = p
        xp = np.where(pos, np.power(np.where(pos, x, 1.0), pw), 1.0 if pw == 0 else 0.0)
        e = np.exp(-b * x)
        return np.stack([xp * e, a * xp * logx * e, -a * x * xp * e])
    raise ValueError(f"no parameter derivatives for kernel kind {spec.kind!r}")


def quantise(w: np.ndarray, delta: float) -> np.ndarray:
    """q_e = max(1, round(w_e / delta)), round half to even (Appendix
    "Distance quantization", definition of q_e)."""
    return np.maximum(1, np.rint(np.asarray(w, dtype=np.float64) / delta)).astype(np.int64)
