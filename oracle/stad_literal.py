"""Literal StAd-TFI in FP64 — ORACLE, test infrastructure only.

Follows the paper's algorithms in their order and notation, on the quantised
metric: every edge has an integer length q_e >= 1 (Appendix "Distance
quantization"), so depths d(u), the backbone coordinate and the table sizes
are in grid units. With unit lengths this is exactly the unweighted
algorithm of Section 2.

Readings where the paper is silent (each also listed in the design notes):
* backbone axis on a weighted tree = grid coordinate X_t = dhat(p_1, p_t);
  the table has L+1 columns, L = X_m (this equals subdividing every edge into
  q_e unit edges whose inner vertices carry no mass);
* diameter = weighted (grid) diameter; first traversal starts at the smallest
  vertex id of S, farthest vertex ties -> smallest id; p_1 is the first
  farthest vertex, p_m the vertex farthest from it;
* centroid = smallest id among vertices whose removal leaves components of at
  most |V(S)|/2 vertices;
* score (Eq. "stad-score") with M = (H+1)(L+1), H, L, H_alpha in grid units,
  n_alpha in vertices, natural log; the centroid wins only if strictly smaller;
* an optional leaf cutoff s0: calls with |V(S)| <= s0 are summed directly
  (s0 = 1 is the paper's base case f(0) x_u).
"""
from __future__ import annotations

import math
from collections import deque

import numpy as np

from .kernels import grid_table, quantise


class Graph:
    """Adjacency lists (neighbours ascending) with quantised lengths."""

    def __init__(self, tree, delta: float):
        self.n = tree.n
        q = quantise(tree.w, delta)
        self.nbrs = [[] for _ in range(tree.n)]
        for a, b, l in zip(tree.u.tolist(), tree.v.tolist(), q.tolist()):
            self.nbrs[a].append((b, l))
            self.nbrs[b].append((a, l))
        for lst in self.nbrs:
            lst.sort()

    def distances(self, src: int, inside: set):
        """Grid distances and parents from src over the vertex set `inside`."""
        dist = {src: 0}
        par = {src: -1}
        dq = deque([src])
        while dq:
            a = dq.popleft()
            for b, l in self.nbrs[a]:
                if b in inside and b not in dist:
                    dist[b] = dist[a] + l
                    par[b] = a
                    dq.append(b)
        return dist, par


# ---------------------------------------------------------------------------
# Algorithm 1: DecomposeOffPathComponents(S, P)
# ---------------------------------------------------------------------------

def decompose_off_path_components(g: Graph, S: set, P: list):
    on_p = {p: j for j, p in enumerate(P)}
    # backbone coordinates (grid units) and pi(p_j) = p_j, d(p_j) = 0
    X = [0]
    for j in range(1, len(P)):
        X.append(X[-1] + dict(g.nbrs[P[j - 1]])[P[j]])
    pi = {p: p for p in P}
    d = {p: 0 for p in P}
    comps = []
    # scan backbone adjacency lists, each off-path neighbour roots a component
    for j, p in enumerate(P):
        for r, l in g.nbrs[p]:
            if r in S and r not in on_p:
                # BFS from r inside S \ P; ell(u) = distance from r
                verts = [r]
                dist = {r: 0}
                dq = deque([r])
                while dq:
                    a = dq.popleft()
                    for b, lb in g.nbrs[a]:
                        if b in S and b not in on_p and b not in dist:
                            dist[b] = dist[a] + lb
                            verts.append(b)
                            dq.append(b)
                h = 0
                for u in verts:
                    pi[u] = p
                    d[u] = dist[u] + l  # the attaching edge p - r adds its length
                    h = max(h, d[u])
                comps.append(dict(root=r, anchor=j, verts=verts, H=h))
    H = max([0] + [c["H"] for c in comps])
    return dict(P=list(P), X=X, pi=pi, d=d, H=H, comps=comps)


# ---------------------------------------------------------------------------
# Algorithm 6: ChooseBackbone(S) and Eq. "stad-score"
# ---------------------------------------------------------------------------

def diameter_path(g: Graph, S: set):
    s0 = min(S)
    dist, _ = g.distances(s0, S)
    a = min(S, key=lambda v: (-dist[v], v))
    dist, par = g.distances(a, S)
    b = min(S, key=lambda v: (-dist[v], v))
    path = [b]
    while path[-1] != a:
        path.append(par[path[-1]])
    path.reverse()
    return path


def centroid(g: Graph, S: set):
    n = len(S)
    root = min(S)
    _, par = g.distances(root, S)
    # children lists and subtree sizes by reverse BFS order
    order = [root]
    i = 0
    while i < len(order):
        a = order[i]
        i += 1
        for b, _ in g.nbrs[a]:
            if b in S and par.get(b) == a:
                order.append(b)
    size = {v: 1 for v in S}
    for v in reversed(order):
        if par[v] >= 0:
            size[par[v]] += size[v]
    best = None
    for v in sorted(S):
        biggest = n - size[v]
        for b, _ in g.nbrs[v]:
            if b in S and par.get(b) == v:
                biggest = max(biggest, size[b])
        if 2 * biggest <= n:
            best = v
            break
    return best


def score(nS: int, dec) -> float:
    M = (dec["H"] + 1) * (dec["X"][-1] + 1)
    c = float(nS) + M * math.log(max(M, 2))
    for comp in dec["comps"]:
        c += comp["H"] * math.log(comp["H"] + 1)
    for comp in dec["comps"]:
        nA = len(comp["verts"])
        c += nA * math.log(nA + 1)
    return c


def choose_backbone(g: Graph, S: set, policy: str = "adaptive"):
    if policy == "diameter":
        P = diameter_path(g, S)
        return P, decompose_off_path_components(g, S, P), "diameter"
    if policy == "centroid":
        P = [centroid(g, S)]
        return P, decompose_off_path_components(g, S, P), "centroid"
    Pd = diameter_path(g, S)
    Pc = [centroid(g, S)]
    dd = decompose_off_path_components(g, S, Pd)
    dc = decompose_off_path_components(g, S, Pc)
    if score(len(S), dc) < score(len(S), dd):
        return Pc, dc, "centroid"
    return Pd, dd, "diameter"  # diameter wins ties


# ---------------------------------------------------------------------------
# Eq. "sumofFFTterms" evaluators: direct loop, Algorithm 2, Algorithm 3, and
# the Hankel-matrix product with antidiagonal prefix sums
# ---------------------------------------------------------------------------

def compute_g_direct(A: np.ndarray, fv: np.ndarray) -> np.ndarray:
    """Four nested loops over (q, s, r, t) as in the proof of the 1D-FFT proposition."""
    H1, W = A.shape[:2]
    G = np.zeros_like(A)
    for q in range(H1):
        for s in range(W):
            for r in range(H1):
                for t in range(W):
                    G[q, s] += fv[q + r + abs(s - t)] * A[r, t]
    return G


def _pow2(n: int) -> int:
    return 1 << max(0, (n - 1).bit_length())


def compute_g_1d(A: np.ndarray, fv: np.ndarray) -> np.ndarray:
    """Algorithm 2: one zero-padded 1D convolution per depth pair (q, r)."""
    H1, W = A.shape[:2]
    L = _pow2(3 * W - 2)
    G = np.zeros_like(A)
    j = np.arange(2 * W - 1)
    for q in range(H1):
        for r in range(H1):
            a = A[r]
            b = fv[q + r + np.abs(j - (W - 1))]
            y = np.fft.irfft(np.fft.rfft(a, L, axis=0) * np.fft.rfft(b, L)[:, None], L, axis=0)
            G[q] += y[W - 1: 2 * W - 1]
    return G


def compute_g_2dfft(A: np.ndarray, fv: np.ndarray) -> np.ndarray:
    """Algorithm 3: depth reversal, 2D kernel, one 2D FFT convolution, crop.

    A: (H+1, W, d) aggregates. fv: f at grid distances 0.. >= 2H + W - 1.
    """
    H1, W, d = A.shape
    H = H1 - 1
    Abar = A[::-1]                                     # Abar[rho, j] = A_{H - rho}[j]
    i = np.arange(2 * H + 1)[:, None]
    j = np.arange(2 * W - 1)[None, :]
    Kbar = fv[i + np.abs(j - (W - 1))]                 # Kbar[i, j] = f(i + |j - (W-1)|)
    s = (_pow2(3 * H + 1), _pow2(3 * W - 2))
    KF = np.fft.rfft2(Kbar, s)
    AF = np.fft.rfft2(Abar, s, axes=(0, 1))
    Y = np.fft.irfft2(AF * KF[:, :, None], s, axes=(0, 1))
    return Y[H: 2 * H + 1, W - 1: 2 * W - 1]           # G_q[s] = Y[q + H, s + W - 1]


def _left_offsets(B: np.ndarray, H1: int) -> np.ndarray:
    """L_q[s] = sum_{t <= s} B[q + s - t, t]: every term lies on the
    antidiagonal sigma = l + t = q + s, so an inclusive running sum over t
    along each antidiagonal, read at t = s, gives it."""
    nl, W = B.shape[:2]
    out = np.zeros((H1, W) + B.shape[2:])
    for sigma in range(nl + W - 1):
        run = np.zeros(B.shape[2:])
        for t in range(W):
            l = sigma - t
            if l < 0:
                break
            if l < nl:
                run = run + B[l, t]
            q = sigma - t  # reading at s = t
            if q < H1:
                out[q, t] = run
    return out


def compute_g_hankel(A: np.ndarray, fv: np.ndarray) -> np.ndarray:
    """Attention-width evaluation of Eq. "sumofFFTterms" (appendix on the
    cross term at attention width): with l = q + |s - t| the kernel argument
    is l + r, so first the depth correlation B[l, t] = sum_r f(l + r) A_r[t]
    for l = 0 .. H + m - 1 as ONE matrix product with the Hankel matrix
    F[l, r] = f(l + r) of shape (H + m) x (H + 1) and A reshaped to
    (H + 1) x (m d); then G_q[s] = sum_t B[q + |s - t|, t] split at t = s into
    a left part (prefix sums along antidiagonals), a right part (the same on
    the reversed backbone) and minus B[q, s], counted in both.

    A: (H+1, m, d) aggregates. fv: f at grid distances 0 .. >= 2H + m - 1.
    """
    H1, W, d = A.shape
    nl = H1 - 1 + W
    Fh = fv[np.arange(nl)[:, None] + np.arange(H1)[None, :]]          # Hankel: depends on l + r only
    B = (Fh @ A.reshape(H1, W * d)).reshape(nl, W, d)                  # one GEMM for all t and channels
    left = _left_offsets(B, H1)
    right = _left_offsets(B[:, ::-1], H1)[:, ::-1]                     # reversed backbone direction
    return left + right - B[:H1]


def compute_e_fft(b: np.ndarray, fv: np.ndarray) -> np.ndarray:
    """E[q] = sum_{r>=1} f(q + r) b[r], q = 0..H_alpha (Eq. "stad-E"), by a
    zero-padded 1D FFT after reversing the profile. b[0] = 0."""
    Ha = b.shape[0] - 1
    brev = b[::-1]
    fseq = fv[: 2 * Ha + 1]
    L = _pow2(3 * Ha + 1)
    y = np.fft.irfft(np.fft.rfft(brev, L, axis=0) * np.fft.rfft(fseq, L)[:, None], L, axis=0)
    return y[Ha: 2 * Ha + 1]


# ---------------------------------------------------------------------------
# Cross-component term of Eq. "stad-split" (Lemma "Cross-component correction")
# ---------------------------------------------------------------------------

def _vertex_coords(dec):
    """Per vertex of S: depth d(u), backbone column X(pi(u)) and component
    index (-1 on the backbone), as three aligned arrays plus the vertex ids."""
    col_of = {p: dec["X"][j] for j, p in enumerate(dec["P"])}
    comp_of = {}
    for ci, comp in enumerate(dec["comps"]):
        for u in comp["verts"]:
            comp_of[u] = ci
    verts = np.array(sorted(dec["d"]), dtype=np.int64)
    depth = np.array([dec["d"][u] for u in verts.tolist()], dtype=np.int64)
    col = np.array([col_of[dec["pi"][u]] for u in verts.tolist()], dtype=np.int64)
    cid = np.array([comp_of.get(u, -1) for u in verts.tolist()], dtype=np.int64)
    return verts, depth, col, cid


def cross_subroutine(dec, x: np.ndarray, fv: np.ndarray, evaluator: str = "fft2d"):
    """Cross_P(u) for every u in S (Lemma "Cross-component correction").

    By Lemma "Distances through the backbone", a source v outside u's
    component is at distance d(u) + |X(pi u) - X(pi v)| + d(v), so summing
    f over all of S with that surrogate distance is the table
    G_q[s] = sum_{r,t} f(q + |s - t| + r) A_r[t] of Eq. "sumofFFTterms",
    A being the field binned by (depth, backbone column). The surrogate is
    wrong exactly for sources in u's own component, whose surrogate
    distance is d(u) + d(v); their total is E_alpha[d(u)] of Eq. "stad-E"
    (sources at depth >= 1 only, since every vertex of a component has
    depth >= 1). So Cross(u) = G[d(u), X(pi u)] - E_alpha(u)[d(u)], with no
    correction on the backbone.
    """
    H, W, d = dec["H"], dec["X"][-1] + 1, x.shape[1]
    verts, depth, col, cid = _vertex_coords(dec)
    A = np.zeros((H + 1, W, d))
    np.add.at(A, (depth, col), x[verts])
    G = {"fft2d": compute_g_2dfft, "fft1d": compute_g_1d, "hankel": compute_g_hankel}.get(
        evaluator, compute_g_direct)(A, fv)
    out = G[depth, col].copy()
    Es = []
    for ci, comp in enumerate(dec["comps"]):
        mine = cid == ci
        b = np.zeros((comp["H"] + 1, d))
        np.add.at(b, depth[mine], x[verts[mine]])
        E = compute_e_fft(b, fv)
        Es.append(E)
        out[mine] -= E[depth[mine]]
    return {int(u): out[i] for i, u in enumerate(verts.tolist())}, dict(A=A, G=G, E=Es)


# ---------------------------------------------------------------------------
# Algorithm 7: CrossSubRoutineExp(S, P, x, f) for f(k) = sum_l c_l lambda_l^k
# ---------------------------------------------------------------------------

def cross_subroutine_exp(dec, x: np.ndarray, terms):
    """Two backbone sweeps per exponential term. On grid units consecutive
    backbone vertices are q_s apart, so the sweep factors are lambda^{q_s}
    (the weighted form the paper uses for its diameter variant)."""
    P, X = dec["P"], dec["X"]
    m = len(P)
    d = x.shape[1]
    cross = {u: np.zeros(d) for u in dec["d"]}
    index_of = {p: s for s, p in enumerate(P)}
    for c, lam in terms:
        G0 = np.zeros((m, d))
        for u, du in dec["d"].items():
            G0[index_of[dec["pi"][u]]] += lam ** du * x[u]
        E0 = []
        for comp in dec["comps"]:
            E0.append(sum(lam ** dec["d"][u] * x[u] for u in comp["verts"]))
        for s in range(1, m):                                # forward sweep
            G0[s] = G0[s] + lam ** (X[s] - X[s - 1]) * G0[s - 1]
        for s in range(m - 2, -1, -1):                       # backward sweep
            g = lam ** (X[s + 1] - X[s])
            G0[s] = (1.0 - g * g) * G0[s] + g * G0[s + 1]
        for s, p in enumerate(P):
            cross[p] = cross[p] + c * G0[s]
        for comp, e0 in zip(dec["comps"], E0):
            a = comp["anchor"]
            for u in comp["verts"]:
                cross[u] = cross[u] + c * lam ** dec["d"][u] * (G0[a] - e0)
    return cross


# ---------------------------------------------------------------------------
# Algorithm 5: Solve(S, x, f)
# ---------------------------------------------------------------------------

class Result:
    def __init__(self):
        self.calls = []   # non-leaf calls: dict(level, minv, size, kind, P, X, rec)
        self.leaves = []  # dict(level, minv, size, verts)


def solve(tree, delta: float, spec, x, policy: str = "adaptive", leaf_max: int = 1,
          evaluator: str = "fft2d", exp_terms=None, evaluate: bool = True):
    """Returns (w, Result). x: (n,) or (n, d). With exp_terms = [(c, lambda)]
    per grid unit, the cross terms use Algorithm 7 instead of FFTs. With
    evaluate=False only the decomposition is recorded (w stays zero)."""
    g = Graph(tree, delta)
    x = np.asarray(x, dtype=np.float64)
    squeeze = x.ndim == 1
    if squeeze:
        x = x[:, None]
    n, d = x.shape
    # f on the grid, long enough for every lookup the algorithms make
    from .brute import Adjacency
    kmax = 3 * Adjacency(tree, delta).max_dist() + 4 if evaluate else 0
    fv = grid_table(spec, delta, kmax) if spec.kind != "table" else _padded_table(spec, kmax)
    w = np.zeros((n, d))
    res = Result()
    # top-level calls: the trees of the forest
    seen = np.zeros(n, dtype=bool)
    stack = []
    for s in range(n):
        if not seen[s]:
            comp, _ = g.distances(s, _All())
            for v in comp:
                seen[v] = True
            stack.append((0, set(comp)))
    while stack:
        level, S = stack.pop()
        if len(S) <= leaf_max:
            verts = sorted(S)
            for u in (verts if evaluate else []):
                du, _ = g.distances(u, S)
                w[u] += sum(fv[du[v]] * x[v] for v in verts)
            res.leaves.append(dict(level=level, minv=verts[0], size=len(S), verts=verts))
            continue
        P, dec, kind = choose_backbone(g, S, policy)
        if not evaluate:
            cross, inter = {u: 0.0 for u in S}, None
        elif exp_terms is not None:
            cross = cross_subroutine_exp(dec, x, exp_terms)
            inter = None
        else:
            cross, inter = cross_subroutine(dec, x, fv, evaluator)
        for u in S:
            w[u] += cross[u]
        rec = {}
        col_of = {p: dec["X"][j] for j, p in enumerate(P)}
        for ci, comp in enumerate(dec["comps"]):
            cmin = min(comp["verts"])
            for u in comp["verts"]:
                rec[u] = (dec["d"][u], col_of[dec["pi"][u]], cmin)
        for p in P:
            rec[p] = (0, col_of[p], -1)
        res.calls.append(dict(level=level, minv=min(S), size=len(S), kind=kind, P=list(P), X=list(dec["X"]),
                              H=dec["H"], comps=[(min(c["verts"]), c["anchor"], c["H"], len(c["verts"]))
                                                 for c in dec["comps"]],
                              rec=rec, inter=inter))
        for comp in dec["comps"]:
            stack.append((level + 1, set(comp["verts"])))
    return (w[:, 0] if squeeze else w), res


class _All:
    def __contains__(self, v):
        return True


def _padded_table(spec, kmax):
    t = np.asarray(spec.table, dtype=np.float64)
    out = np.zeros(kmax + 1)
    out[: min(t.shape[0], kmax + 1)] = t[: kmax + 1]
    return out
