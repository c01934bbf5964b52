"""Kernel specifications f(x) of a distance x (original units).

A spec is a kind plus parameters; it holds no evaluation code. Kinds:

* ``expsum``   f(x) = sum_k a_k exp(-b_k x),        params [a_1, b_1, a_2, b_2, ...]
* ``gauss``    f(x) = a exp(-c x^2),                params [a, c]
* ``rational`` f(x) = a / (1 + c x^e)^p,            params [a, c, e, p]
* ``powexp``   f(x) = a x^p exp(-b x),              params [a, p, b]
* ``table``    f(k * delta) = table[k], k = 0..len-1 (samples on the distance grid)
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

KINDS = {"table": 0, "expsum": 1, "gauss": 2, "rational": 3, "powexp": 4}


@dataclass
class KernelSpec:
    kind: str
    params: list = field(default_factory=list)
    table: np.ndarray | None = None

    def __post_init__(self):
        assert self.kind in KINDS, self.kind

    @property
    def kind_id(self) -> int:
        return KINDS[self.kind]

    # named constructors for the kernels used by the benchmark configurations
    @staticmethod
    def exp(lam: float, a: float = 1.0) -> "KernelSpec":
        return KernelSpec("expsum", [a, lam])

    @staticmethod
    def expsum(a, b) -> "KernelSpec":
        p = []
        for ai, bi in zip(a, b):
            p += [float(ai), float(bi)]
        return KernelSpec("expsum", p)

    @staticmethod
    def gauss(c: float, a: float = 1.0) -> "KernelSpec":
        return KernelSpec("gauss", [a, c])

    @staticmethod
    def rational(c: float, e: float = 1.0, p: float = 1.0, a: float = 1.0) -> "KernelSpec":
        return KernelSpec("rational", [a, c, e, p])

    @staticmethod
    def powexp(b: float, p: float = 1.0, a: float = 1.0) -> "KernelSpec":
        return KernelSpec("powexp", [a, p, b])

    @staticmethod
    def samples(table) -> "KernelSpec":
        return KernelSpec("table", [], np.asarray(table, dtype=np.float64))
