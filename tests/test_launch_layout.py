"""Host-side launch layouts of a plan (no GPU): the packing of big dense leaves
into CTAs of the big-leaf kernel, and the vertex order of the output gather.
Neither changes what is computed; these tests check that every piece of work is
scheduled exactly once and within the kernels' limits."""
import numpy as np
import pytest

import workloads as W

from ._lib import tfi

WARPS, PER_WARP, BIG = 8, 64, 64


def _plans():
    out = []
    for shape, n, s0 in [("rrt", 1 << 14, 512), ("caterpillar", 1 << 12, 256), ("binary", 1 << 13, 128)]:
        cfg = W.configs.sweep(shape, n=n, d=16)
        out.append((f"{shape}_{n}_s0{s0}", cfg["tree"], cfg["delta"], cfg["kernel"], s0))
    cfg = W.configs.uneven_batch(count=30, lo=8, hi=3000, d=16)
    out.append(("forest30", cfg["tree"], cfg["delta"], cfg["kernel"], 512))
    return out


PLANS = _plans()


@pytest.mark.parametrize("name,tree,delta,spec,s0", PLANS, ids=[p[0] for p in PLANS])
def test_big_leaves_packed_once_within_limits(name, tree, delta, spec, s0):
    p = tfi.Plan.from_spec(tree, delta, spec, leaf_max=s0, host_only=True)
    sizes = p.export("leaves")[:, 2]
    ends = np.cumsum(sizes)
    ranges = {(int(e - s), int(e)) for s, e in zip(sizes, ends) if s >= BIG}
    packs = p.export("leaf_packs")
    if not ranges:
        assert packs.size == 0
        return
    got = [(int(b), int(e)) for b, e in packs[:, 1:3]]
    assert len(got) == len(set(got)) == len(ranges) and set(got) == ranges
    cap = int(packs[0, 3])
    assert (packs[:, 3] == cap).all()
    assert cap >= max(e - b for b, e in ranges) and cap >= WARPS * PER_WARP
    ctas = packs[:, 0]
    assert (np.diff(ctas) >= 0).all() and (np.diff(np.unique(ctas)) == 1).all() and ctas[0] == 0
    first = []
    for c in np.unique(ctas):
        rows = packs[ctas == c]
        n = rows[:, 2] - rows[:, 1]
        first.append(int(n[0]))
        if len(rows) > 1:
            assert int(np.minimum(WARPS, (n + PER_WARP - 1) // PER_WARP).sum()) <= WARPS
            assert int(n.sum()) <= cap
            assert (n <= WARPS * PER_WARP).all()
    # CTAs are opened largest leaf first
    assert all(a >= b for a, b in zip(first, first[1:]))


def _tc_cost(n):
    # work of one leaf in the persistent tensor-core leaf kernel: 128-row tiles x 32-source chunks + 4
    return -(-n // 128) * -(-n // 32) + 4


@pytest.mark.parametrize("name,tree,delta,spec,s0", PLANS, ids=[p[0] for p in PLANS])
def test_tensor_core_leaves_dealt_longest_first(name, tree, delta, spec, s0):
    """Every big leaf goes to exactly one persistent CTA; each CTA's list runs largest first; the
    greedy longest-first assignment keeps every CTA within one leaf's work of the least-loaded one
    and within 4/3 of the lower bound on the best makespan."""
    p = tfi.Plan.from_spec(tree, delta, spec, leaf_max=s0, host_only=True)
    sizes = p.export("leaves")[:, 2]
    ends = np.cumsum(sizes)
    ranges = sorted((int(e - s), int(e)) for s, e in zip(sizes, ends) if s >= BIG)
    rows = p.export("leaf_ctas")
    if not ranges:
        assert rows.size == 0
        return
    got = sorted((int(b), int(e)) for b, e in rows[:, 1:3])
    assert got == ranges
    n_ctas = int(rows[0, 3])
    assert (rows[:, 3] == n_ctas).all() and 1 <= n_ctas <= len(ranges)
    cta = rows[:, 0]
    assert (np.diff(cta) >= 0).all() and set(cta.tolist()) == set(range(n_ctas))
    load = np.zeros(n_ctas)
    for c in range(n_ctas):
        n = rows[cta == c, 2] - rows[cta == c, 1]
        assert (np.diff(n) <= 0).all()
        load[c] = sum(_tc_cost(int(x)) for x in n)
    costs = [_tc_cost(e - b) for b, e in ranges]
    assert load.max() - load.min() <= max(costs) + 1e-9
    bound = max(sum(costs) / n_ctas, max(costs))
    assert load.max() <= 4.0 / 3.0 * bound + 1e-9


def _is_dfs_preorder(order, n, u, v):
    adj = [[] for _ in range(n)]
    for a, b in zip(u, v):
        adj[a].append(b)
        adj[b].append(a)
    adjs = [set(x) for x in adj]
    seen = np.zeros(n, dtype=bool)
    stack = []
    for w in order:
        w = int(w)
        if seen[w]:
            return False
        while stack and w not in adjs[stack[-1]]:
            stack.pop()
        if not stack:
            # a new tree starts at its smallest vertex, none of its neighbours seen
            if any(seen[x] for x in adj[w]) or (seen[:w] == False).any():  # noqa: E712
                return False
        seen[w] = True
        stack.append(w)
    return bool(seen.all())


@pytest.mark.parametrize("name,tree,delta,spec,s0", PLANS, ids=[p[0] for p in PLANS])
def test_gather_order_is_a_depth_first_preorder(name, tree, delta, spec, s0):
    p = tfi.Plan.from_spec(tree, delta, spec, leaf_max=s0, host_only=True)
    order = p.export("gather_order")
    assert order.shape == (tree.n,)
    assert np.array_equal(np.sort(order), np.arange(tree.n))
    assert _is_dfs_preorder(order, tree.n, np.asarray(tree.u), np.asarray(tree.v))


def test_dfs_check_rejects_a_non_preorder():
    # path 0-1-2 plus leaf 3 on 0: [0, 1, 3, 2] jumps back before finishing 1's subtree
    u, v = np.array([0, 1, 0]), np.array([1, 2, 3])
    assert _is_dfs_preorder([0, 1, 2, 3], 4, u, v)
    assert _is_dfs_preorder([0, 3, 1, 2], 4, u, v)
    assert not _is_dfs_preorder([0, 1, 3, 2], 4, u, v)
    assert not _is_dfs_preorder([1, 0, 2, 3], 4, u, v)
