"""FP64 Sinkhorn on the tree metric — ORACLE, test infrastructure only.

Plain definition with a dense kernel matrix (small trees only): K = f(delta *
dhat) from all-pairs grid distances, then the alternating scalings of the
paper's Sinkhorn driver (Appendix "Sinkhorn Implementation Details", Eq.
"app-sinkhorn-updates"): u = a / (K v + delta), v = b / (K^T u + delta),
u = v = 1 at start. Transport cost of the plan diag(u) K diag(v): sum_ij u_i
K_ij D_ij v_j, i.e. sum_i u_i (K2 v)_i with K2 = f2(delta * dhat),
f2(x) = x exp(-x / eps).
"""
from __future__ import annotations

import numpy as np

from .brute import Adjacency
from .kernels import grid_table


def dense_matrix(tree, delta: float, spec) -> np.ndarray:
    adj = Adjacency(tree, delta)
    D = adj.dist_rows(np.arange(tree.n))
    if np.any(D < 0):
        raise ValueError("dense_matrix needs a connected tree")
    return grid_table(spec, delta, int(D.max()))[D]


def sinkhorn(K: np.ndarray, a: np.ndarray, b: np.ndarray, iters: int, delta_reg: float = 1e-30):
    u = np.ones_like(a, dtype=np.float64)
    v = np.ones_like(b, dtype=np.float64)
    for _ in range(iters):
        u = a / (K @ v + delta_reg)
        v = b / (K.T @ u + delta_reg)
    return u, v


def transport_cost(K2: np.ndarray, u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Per marginal pair (column): sum_i u_i (K2 v)_i."""
    return np.einsum("ic,ic->c", u, K2 @ v)
