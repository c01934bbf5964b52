"""Seeded fields on tree vertices."""
from __future__ import annotations

import numpy as np


def normal_field(n: int, d: int, seed: int = 123, dtype=np.float32) -> np.ndarray:
    """i.i.d. N(0,1) field of shape (n, d), row-major. Seed 123 follows the
    paper's synthetic protocol (NumPy default_rng(123))."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, d)).astype(dtype)


def dirichlet_pairs(n: int, pairs: int, seed: int = 0, dtype=np.float32):
    """`pairs` source/target marginals, each Dirichlet(1) on n vertices.
    Returns (a, b) of shape (n, pairs)."""
    rng = np.random.default_rng(seed)
    a = np.ascontiguousarray(rng.dirichlet(np.ones(n), size=pairs).T)
    b = np.ascontiguousarray(rng.dirichlet(np.ones(n), size=pairs).T)
    return a.astype(dtype), b.astype(dtype)
