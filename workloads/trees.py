"""Tree and forest generators.

A tree is returned as an edge list ``(u[i], v[i], w[i])`` over vertices
``0..n-1``. Generators of topologies return unit weights; weight helpers at the
bottom draw seeded edge lengths. Families follow the paper's synthetic
benchmark definitions (Appendix "Tree construction and parameter ranges",
Table "Deterministic tree constructions" and the three random constructions
listed under it) and the five benchmark configurations of this project.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np


@dataclass
class Tree:
    """Undirected weighted forest on vertices 0..n-1 (n-1 edges for a tree)."""

    n: int
    u: np.ndarray  # int32 [m]
    v: np.ndarray  # int32 [m]
    w: np.ndarray  # float64 [m], > 0

    @property
    def m(self) -> int:
        return int(self.u.shape[0])

    def with_weights(self, w) -> "Tree":
        w = np.asarray(w, dtype=np.float64)
        assert w.shape == (self.m,)
        return Tree(self.n, self.u, self.v, w)

    def relabel(self, perm) -> "Tree":
        """Return the same forest with vertex i renamed perm[i]."""
        perm = np.asarray(perm, dtype=np.int64)
        return Tree(self.n, perm[self.u].astype(np.int32), perm[self.v].astype(np.int32), self.w.copy())


def _from_parents(parent: np.ndarray) -> Tree:
    """Edges (parent[i], i) for every i with parent[i] >= 0."""
    parent = np.asarray(parent, dtype=np.int64)
    child = np.nonzero(parent >= 0)[0]
    u = parent[child].astype(np.int32)
    v = child.astype(np.int32)
    return Tree(int(parent.shape[0]), u, v, np.ones(u.shape[0]))


def _from_edges(n: int, edges) -> Tree:
    e = np.asarray(list(edges), dtype=np.int64).reshape(-1, 2)
    return Tree(n, e[:, 0].astype(np.int32), e[:, 1].astype(np.int32), np.ones(e.shape[0]))


# --- deterministic families (paper Table "Deterministic tree constructions") ---

def path(n: int) -> Tree:
    parent = np.arange(-1, n - 1)
    return _from_parents(parent)


def star(n: int) -> Tree:
    parent = np.zeros(n, dtype=np.int64)
    parent[0] = -1
    return _from_parents(parent)


def spider(k: int, arm: int) -> Tree:
    """Hub 0 with k arms of `arm` edges each: n = 1 + k*arm."""
    edges = []
    nxt = 1
    for _ in range(k):
        prev = 0
        for _ in range(arm):
            edges.append((prev, nxt))
            prev = nxt
            nxt += 1
    return _from_edges(nxt, edges)


def _spine_with(ell: int, attach) -> Tree:
    """Spine 0..ell-1 (a path) with `attach(t)` pendant structures per spine vertex.

    attach(t) returns a list of chain lengths; each chain hangs off spine vertex t.
    """
    edges = [(t - 1, t) for t in range(1, ell)]
    nxt = ell
    for t in range(ell):
        for length in attach(t):
            prev = t
            for _ in range(length):
                edges.append((prev, nxt))
                prev = nxt
                nxt += 1
    return _from_edges(nxt, edges)


def caterpillar_leaves(ell: int, leaves: int = 3) -> Tree:
    """Spine of ell vertices with `leaves` leaves per spine vertex (n = (leaves+1)*ell)."""
    return _spine_with(ell, lambda t: [1] * leaves)


def caterpillar_hanging_paths(ell: int) -> Tree:
    """Spine of ell vertices, one ell-edge path at each spine vertex (n = ell + ell^2)."""
    return _spine_with(ell, lambda t: [ell])


def toothed_spine(ell: int, h: int, teeth: int = 2) -> Tree:
    """Spine of ell vertices with `teeth` chains of h edges at each spine vertex
    (n = ell (1 + teeth h)): dense two-dimensional bin tables of depth h."""
    return _spine_with(ell, lambda t: [h] * teeth)


def comb(ell: int) -> Tree:
    return caterpillar_leaves(ell, leaves=2)


def broom(ell: int) -> Tree:
    """Handle of ell vertices with ell/2 leaves at one endpoint (n = 3*ell/2)."""
    return _spine_with(ell, lambda t: [1] * (ell // 2) if t == ell - 1 else [])


def double_broom(ell: int) -> Tree:
    """Handle of ell vertices with ell/4 leaves at each endpoint (n = 3*ell/2)."""
    return _spine_with(ell, lambda t: [1] * (ell // 4) if t in (0, ell - 1) else [])


def complete_kary(k: int, depth: int) -> Tree:
    n = (k ** (depth + 1) - 1) // (k - 1)
    i = np.arange(n)
    parent = np.where(i == 0, -1, (i - 1) // k)
    return _from_parents(parent)


def complete_binary_n(n: int) -> Tree:
    """Heap-indexed binary tree on exactly n vertices (last level partially filled)."""
    i = np.arange(n)
    parent = np.where(i == 0, -1, (i - 1) // 2)
    return _from_parents(parent)


# --- random families ---

def random_recursive(n: int, rng: np.random.Generator) -> Tree:
    """Vertex i >= 1 attaches to a uniform vertex of {0..i-1}."""
    i = np.arange(n, dtype=np.float64)
    parent = np.floor(rng.random(n) * i).astype(np.int64)
    parent[0] = -1
    return _from_parents(parent)


def caterpillar_rrt(n: int, rng: np.random.Generator) -> Tree:
    """Path 0..n/4-1, then every vertex i >= n/4 picks a uniform parent in {0..i-1}."""
    spine = max(1, n // 4)
    i = np.arange(n, dtype=np.float64)
    parent = np.floor(rng.random(n) * i).astype(np.int64)
    parent[:spine] = np.arange(-1, spine - 1)
    return _from_parents(parent)


def random_mst_topology(n: int, rng: np.random.Generator) -> Tree:
    """Kruskal MST of the complete graph with iid U[0,1) weights (unit weights kept)."""
    iu, iv = np.triu_indices(n, k=1)
    w = rng.random(iu.shape[0])
    order = np.argsort(w, kind="stable")
    edges = _kruskal(n, iu[order], iv[order])
    return _from_edges(n, edges)


def preferential_attachment(n: int, rng: np.random.Generator) -> Tree:
    """Sampling list starts as [0]; new vertex i picks a parent from the list, then
    appends the parent and itself."""
    lst = [0]
    parent = np.full(n, -1, dtype=np.int64)
    for i in range(1, n):
        p = lst[int(rng.integers(0, len(lst)))]
        parent[i] = p
        lst.append(p)
        lst.append(i)
    return _from_parents(parent)


def _kruskal(n: int, us, vs):
    par = list(range(n))

    def find(a):
        while par[a] != a:
            par[a] = par[par[a]]
            a = par[a]
        return a

    out = []
    for a, b in zip(us.tolist(), vs.tolist()):
        ra, rb = find(a), find(b)
        if ra != rb:
            par[ra] = rb
            out.append((a, b))
            if len(out) == n - 1:
                break
    return out


def torus_knn_mst(n: int, rng: np.random.Generator, R: float = 1.0, r: float = 0.3, k: int = 8) -> Tree:
    """Points area-uniform on a torus surface, symmetrised kNN graph with
    Euclidean weights, minimum spanning tree (components bridged by their
    shortest connecting edges before Kruskal)."""
    from scipy.spatial import cKDTree
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import minimum_spanning_tree, connected_components

    # rejection sampling: the area element is proportional to (R + r cos phi)
    theta = np.empty(0)
    phi = np.empty(0)
    while theta.shape[0] < n:
        m = 2 * (n - theta.shape[0]) + 64
        th = rng.random(m) * 2 * np.pi
        ph = rng.random(m) * 2 * np.pi
        keep = rng.random(m) * (R + r) < (R + r * np.cos(ph))
        theta = np.concatenate([theta, th[keep]])
        phi = np.concatenate([phi, ph[keep]])
    theta, phi = theta[:n], phi[:n]
    pts = np.stack([(R + r * np.cos(phi)) * np.cos(theta),
                    (R + r * np.cos(phi)) * np.sin(theta),
                    r * np.sin(phi)], axis=1)
    kd = cKDTree(pts)
    dist, idx = kd.query(pts, k=k + 1)
    rows = np.repeat(np.arange(n), k)
    cols = idx[:, 1:].reshape(-1)
    d = dist[:, 1:].reshape(-1)
    a = np.minimum(rows, cols)
    b = np.maximum(rows, cols)
    key = a.astype(np.int64) * n + b
    key, first = np.unique(key, return_index=True)
    a, b, d = a[first], b[first], d[first]
    ncomp, lab = connected_components(coo_matrix((d, (a, b)), shape=(n, n)), directed=False)
    while ncomp > 1:
        # bridge each component to its nearest point outside it
        extra_a, extra_b, extra_d = [], [], []
        for c in range(ncomp):
            inside = np.nonzero(lab == c)[0]
            outside = np.nonzero(lab != c)[0]
            kd_out = cKDTree(pts[outside])
            dd, jj = kd_out.query(pts[inside], k=1)
            t = int(np.argmin(dd))
            extra_a.append(inside[t])
            extra_b.append(outside[jj[t]])
            extra_d.append(dd[t])
        a = np.concatenate([a, np.minimum(extra_a, extra_b)])
        b = np.concatenate([b, np.maximum(extra_a, extra_b)])
        d = np.concatenate([d, extra_d])
        ncomp, lab = connected_components(coo_matrix((d, (a, b)), shape=(n, n)), directed=False)
    mst = minimum_spanning_tree(coo_matrix((d, (a, b)), shape=(n, n))).tocoo()
    t = Tree(n, mst.row.astype(np.int32), mst.col.astype(np.int32), mst.data.astype(np.float64))
    assert t.m == n - 1
    return t


def grid_spanning_tree(h: int, w: int, rng: np.random.Generator) -> Tree:
    """Kruskal spanning tree of the h x w grid graph under iid U[0,1] edge
    weights; the returned tree has unit edge lengths."""
    ids = np.arange(h * w).reshape(h, w)
    us = np.concatenate([ids[:, :-1].ravel(), ids[:-1, :].ravel()])
    vs = np.concatenate([ids[:, 1:].ravel(), ids[1:, :].ravel()])
    order = np.argsort(rng.random(us.shape[0]), kind="stable")
    return _from_edges(h * w, _kruskal(h * w, us[order], vs[order]))


def forest(trees) -> tuple[Tree, np.ndarray]:
    """Disjoint union; returns the forest and the vertex offset of each tree."""
    offs = np.zeros(len(trees) + 1, dtype=np.int64)
    for i, t in enumerate(trees):
        offs[i + 1] = offs[i] + t.n
    u = np.concatenate([t.u.astype(np.int64) + offs[i] for i, t in enumerate(trees)])
    v = np.concatenate([t.v.astype(np.int64) + offs[i] for i, t in enumerate(trees)])
    w = np.concatenate([t.w for t in trees])
    return Tree(int(offs[-1]), u.astype(np.int32), v.astype(np.int32), w), offs


def prufer_trees(n: int):
    """Every labelled tree on n >= 2 vertices (n^(n-2) of them), via Pruefer codes."""
    if n == 2:
        yield _from_edges(2, [(0, 1)])
        return
    for code in itertools.product(range(n), repeat=n - 2):
        degree = [1] * n
        for c in code:
            degree[c] += 1
        edges = []
        for c in code:
            leaf = min(i for i in range(n) if degree[i] == 1)
            edges.append((leaf, c))
            degree[leaf] -= 1
            degree[c] -= 1
        a, b = [i for i in range(n) if degree[i] == 1]
        edges.append((a, b))
        yield _from_edges(n, edges)


# --- edge weights ---

def integer_weights(m: int, lo: int, hi: int, rng: np.random.Generator) -> np.ndarray:
    """iid integers uniform on {lo..hi}."""
    return rng.integers(lo, hi + 1, size=m).astype(np.float64)


def snapped_uniform_weights(m: int, lo: float, hi: float, grid: float, rng: np.random.Generator) -> np.ndarray:
    """iid U[lo,hi] snapped to the nearest multiple of `grid` (exact binary
    fractions for grid = 2^-k, so w/grid is an exact integer)."""
    return np.round(rng.uniform(lo, hi, size=m) / grid) * grid


def uniform_weights(m: int, lo: float, hi: float, rng: np.random.Generator) -> np.ndarray:
    return rng.uniform(lo, hi, size=m)
