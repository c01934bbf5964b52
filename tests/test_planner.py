"""Host planner (C++ in libtfi, host-only plans): bit-exact decomposition arrays
against the literal reference, and the paper's structural invariants."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import stad_literal as L

from ._lib import tfi


def _compare(t, delta, spec, policy, s0):
    p = tfi.Plan.from_spec(t, delta, spec, policy=policy, leaf_max=s0, host_only=True)
    calls, bb, recs, leaves = (p.export(k) for k in ("calls", "backbone", "records", "leaves"))
    _, res = L.solve(t, delta, spec, np.zeros(t.n), policy=policy, leaf_max=s0, evaluate=False)
    lit = {(c["minv"], c["size"]): c for c in res.calls}
    assert len(lit) == len(calls)
    off = 0
    for row in calls:
        lev, minv, size, kind, m, H, Lx = row.tolist()
        c = lit[(minv, size)]
        assert c["level"] == lev and (c["kind"] == "centroid") == bool(kind)
        assert bb[off:off + m].tolist() == c["P"]
        assert (c["H"], c["X"][-1]) == (H, Lx)
        off += m
    for ci, v, r, x, cm in recs.tolist():
        c = lit[(calls[ci][1], calls[ci][2])]
        assert c["rec"][v] == (r, x, cm)
    assert sorted(map(tuple, leaves.tolist())) == sorted((l["level"], l["minv"], l["size"]) for l in res.leaves)
    return p


@pytest.mark.parametrize("policy", ["adaptive", "diameter", "centroid"])
@pytest.mark.parametrize("delta", [1.0 / 64, 0.25, 1.0])
def test_bit_exact_against_literal_random(policy, delta):
    for n, seed in [(2, 0), (3, 1), (17, 2), (150, 3), (600, 4)]:
        rng = np.random.default_rng(seed)
        t = W.random_recursive(n, rng)
        t = t.with_weights(W.trees.snapped_uniform_weights(t.m, 0.5, 2.0, 1 / 64, rng))
        for s0 in (1, 8):
            _compare(t, delta, W.KernelSpec.exp(0.1), policy, s0)


@pytest.mark.parametrize("make", [lambda: W.spider(8, 120), lambda: W.caterpillar_hanging_paths(16),
                                  lambda: W.path(300), lambda: W.complete_binary_n(511), lambda: W.star(80),
                                  lambda: W.caterpillar_leaves(40), lambda: W.broom(80), lambda: W.double_broom(80),
                                  lambda: W.complete_kary(3, 5), lambda: W.comb(60),
                                  lambda: W.preferential_attachment(300, np.random.default_rng(1)),
                                  lambda: W.random_mst_topology(120, np.random.default_rng(2))])
def test_bit_exact_against_literal_families(make):
    for policy in ("adaptive", "diameter"):
        _compare(make(), 1.0, W.KernelSpec.rational(1.0), policy, 1)


def test_forest_bit_exact():
    f, _ = W.forest([W.random_recursive(n, np.random.default_rng(n)) for n in (1, 2, 9, 70, 33)])
    _compare(f, 1.0, W.KernelSpec.exp(0.5), "adaptive", 4)


def _stats(p):
    calls = p.export("calls")
    leaves = p.export("leaves")
    return calls, leaves


@pytest.mark.parametrize("make", [lambda: W.random_recursive(3000, np.random.default_rng(5)),
                                  lambda: W.complete_binary_n(4095), lambda: W.caterpillar_hanging_paths(40),
                                  lambda: W.spider(12, 200), lambda: W.preferential_attachment(2000, np.random.default_rng(6))])
def test_structural_invariants_unit_weights(make):
    t = make()
    n = t.n
    p = tfi.Plan.from_spec(t, 1.0, W.KernelSpec.exp(0.3), policy="adaptive", leaf_max=1, host_only=True)
    calls, leaves = _stats(p)
    # sum_S m_S = n (every vertex lies on exactly one backbone; singletons have m = 1)
    assert calls[:, 4].sum() + leaves.shape[0] == n
    # sum_S k_S = |R| - 1: every call except the root is a component of its parent
    info = p.info()
    recs = p.export("records")
    ncomp = len({(c, cm) for c, _, _, _, cm in recs.tolist() if cm >= 0})
    assert ncomp == calls.shape[0] + leaves.shape[0] - 1
    # sum_S |V(S)| <= n log2(n+1) for the adaptive rule (paper, volume bound of the adaptive recursion)
    assert calls[:, 2].sum() + leaves.shape[0] <= n * math.log2(n + 1)
    # M_S = (H+1) m <= (3 + 1/ln 2) |V(S)| for the selected backbone (adaptive selection lemma)
    M = (calls[:, 5] + 1) * calls[:, 4]
    assert np.all(M <= (3 + 1 / math.log(2)) * calls[:, 2] + 1e-9)
    assert info["n_records"] == calls[:, 2].sum()


def test_diameter_backbone_depth_bound():
    # on a diameter backbone with m vertices, every off-path depth is at most (m-1)/2
    t = W.random_recursive(2000, np.random.default_rng(7))
    p = tfi.Plan.from_spec(t, 1.0, W.KernelSpec.exp(0.3), policy="diameter", leaf_max=1, host_only=True)
    calls, _ = _stats(p)
    assert np.all(2 * calls[:, 5] <= calls[:, 4] - 1)


def test_info_counts_consistent():
    t = W.random_recursive(5000, np.random.default_rng(8))
    t = t.with_weights(W.trees.snapped_uniform_weights(t.m, 0.5, 2.0, 1 / 64, np.random.default_rng(9)))
    p = tfi.Plan.from_spec(t, 1 / 64, W.KernelSpec.gauss(1 / 8), policy="adaptive", leaf_max=64, host_only=True)
    info = p.info()
    calls, leaves = _stats(p)
    assert info["n_calls"] == calls.shape[0] and info["n_leaves"] == leaves.shape[0]
    # every vertex ends on exactly one backbone of a non-leaf call or in exactly one leaf
    assert leaves[:, 2].sum() + calls[:, 4].sum() == t.n and np.all(leaves[:, 2] <= 64)
    assert info["n_jobs_fft"] + info["n_jobs_direct"] >= info["n_calls"]


def test_hankel_selection_host_only():
    # TFI_PLAN_HANKEL_ALL: every job within the limits (H + 1 <= 64, H + L + 1 <= 128 grid units)
    # uses the Hankel evaluator; TFI_PLAN_HANKEL: the channel-aware cost model picks it more often
    # with many channels than with one
    cfg = W.configs.attention(heads=1)
    h = cfg["heads"][0]
    mk = lambda **kw: tfi.Plan.from_spec(h["tree"], 1.0, h["kernel"], leaf_max=16, host_only=True, **kw)
    all_ = mk(max_channels=4096, hankel="all").info()
    none = mk(max_channels=4096).info()
    assert all_["n_jobs_hankel"] > 0 and none["n_jobs_hankel"] == 0
    assert all_["n_jobs_hankel"] + all_["n_jobs_direct"] + all_["n_jobs_fft"] == \
        none["n_jobs_direct"] + none["n_jobs_fft"]
    wide = mk(max_channels=4096, hankel="auto").info()["n_jobs_hankel"]
    narrow = mk(max_channels=1, hankel="auto").info()["n_jobs_hankel"]
    assert wide >= narrow
    # grid-unit tables beyond the limits never qualify
    cfg = W.configs.sweep(shape="rrt", n=1 << 12, d=1, kernel="exp")
    big = tfi.Plan.from_spec(cfg["tree"], cfg["delta"], cfg["kernel"], leaf_max=1, host_only=True,
                             hankel="all").info()
    assert big["n_jobs_fft"] + big["n_jobs_direct"] > 0


def test_sweep_auto_selection_host_only():
    # exponential sums: the cost model sends large tables to the sweeps and keeps small ones direct;
    # other kernels never use the sweeps
    cfg = W.configs.sweep(shape="rrt", n=1 << 14, d=16, kernel="exp")
    mk = lambda spec, **kw: tfi.Plan.from_spec(cfg["tree"], cfg["delta"], spec, leaf_max=64, max_channels=16,
                                              host_only=True, **kw).info()
    auto = mk(cfg["kernel"], sweep="auto")
    plain = mk(cfg["kernel"])
    assert auto["n_jobs_sweep"] > 0 and plain["n_jobs_sweep"] == 0
    assert auto["n_jobs_sweep"] + auto["n_jobs_fft"] + auto["n_jobs_direct"] == plain["n_jobs_fft"] + plain["n_jobs_direct"]
    other = mk(W.KernelSpec.rational(1.0), sweep="auto")
    assert other["n_jobs_sweep"] == 0


@pytest.mark.parametrize("policy", ["adaptive", "diameter", "centroid"])
def test_parallel_planning_is_deterministic(policy):
    # the planner decomposes the calls of a level (and the trees of a forest) on all
    # host threads; the plan must not depend on their interleaving
    single = W.configs.sweep("rrt", n=1 << 15, d=16)
    forest = W.configs.uneven_batch(count=50, lo=8, hi=4000, d=16)
    for cfg, s0 in ((single, 64), (forest, 16)):
        exports = []
        for _ in range(3):
            p = tfi.Plan.from_spec(cfg["tree"], cfg["delta"], cfg["kernel"], policy=policy, leaf_max=s0,
                                   host_only=True)
            exports.append({k: p.export(k) for k in ("calls", "backbone", "records", "leaves", "leaf_packs",
                                                      "gather_order")})
        for e in exports[1:]:
            for k in e:
                assert np.array_equal(e[k], exports[0][k]), k


def test_first_invalid_edge_is_reported_across_blocks():
    # edges are validated in parallel blocks; the error names the first invalid edge in
    # input order, as a single pass would
    n = 200_000
    u = np.arange(1, n, dtype=np.int32)
    v = (u - 1).astype(np.int32)
    w = np.ones(n - 1)

    def error(u, v, w):
        with pytest.raises(tfi.TfiError) as e:
            tfi.Plan(n, u, v, w, delta=1.0, kernel=("expsum", [1.0, 1.0]), leaf_max=8, host_only=True)
        return e.value.name, str(e.value)

    w1 = w.copy()
    w1[150_000], w1[70_000] = np.nan, -1.0
    assert error(u, v, w1) == ("WEIGHT", "tfi error WEIGHT: edge 70000 has a weight that is not finite and positive")
    u2, w2 = u.copy(), w.copy()
    u2[140_000], w2[90_000] = n + 5, 0.0
    assert error(u2, v, w2)[1].endswith("edge 90000 has a weight that is not finite and positive")
    u3 = u.copy()
    u3[100] = v[100]
    assert error(u3, v, w1)[0] == "NOT_TREE" and "edge 100 " in error(u3, v, w1)[1]
    w4 = w.copy()
    w4[123_456] = 1e12
    assert error(u, v, w4)[0] == "GRID_OVERFLOW"


@pytest.mark.parametrize("n,edges", [(1, []), (2, [(0, 1)]), (5, [(0, 1), (3, 4)]), (7, []), (3, [(2, 0)])])
@pytest.mark.parametrize("policy", ["adaptive", "diameter", "centroid"])
def test_degenerate_forests_plan_on_the_host(n, edges, policy):
    u = np.array([e[0] for e in edges], dtype=np.int32)
    v = np.array([e[1] for e in edges], dtype=np.int32)
    p = tfi.Plan(n, u, v, np.ones(len(edges)), delta=1.0, kernel=("expsum", [1.0, 1.0]), leaf_max=1,
                 policy=policy, host_only=True)
    assert np.array_equal(np.sort(p.export("gather_order")), np.arange(n))
    assert p.info()["n_calls"] == sum(1 for _ in edges)  # every 2-vertex tree is one call at s0 = 1
