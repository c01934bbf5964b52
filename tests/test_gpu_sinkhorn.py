"""Sinkhorn on the tree metric (Eq. app-sinkhorn-updates): the device driver
(FP32, graph-replayed iterations) against the FP64 dense oracle, on the
torus-MST workload recipe at a size the dense oracle handles.

Two regimes. At eps = 2 the FP64 iteration has converged after 200 steps
(marginal residual ~1e-9), so the transport costs must agree. At eps = 0.5 it
is still moving after 200 steps, where FP32 and FP64 trajectories may part, so
the update rule is checked on a short trajectory instead. At the configured
eps = 0.05 the iteration divides by entries of K v many orders of magnitude
below their maximum: with every table summed directly (TFI_PLAN_DIRECT_ALL;
the support truncation keeps the tables short) each entry keeps its own
relative accuracy, and 200 FP32 iterations reach the FP64 transport cost; the
FFT-table operator is checked normwise."""
import numpy as np
import pytest

import workloads as W
from oracle import sinkhorn as S

from ._lib import tfi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(eps):
    cfg = W.configs.torus_sinkhorn(n=3000, pairs=8)
    t, delta = cfg["tree"], cfg["delta"]
    spec = W.KernelSpec.exp(1.0 / eps)
    a, b = W.dirichlet_pairs(t.n, 8, seed=1)
    plan = tfi.Plan.from_spec(t, delta, spec, leaf_max=256, max_channels=8)
    return t, delta, spec, a, b, plan


def test_sinkhorn_converged_transport_cost_matches_fp64():
    eps = 2.0
    t, delta, spec, a, b, plan = _setup(eps)
    u, v = plan.sinkhorn(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), iters=200)
    K = S.dense_matrix(t, delta, spec)
    uo, vo = S.sinkhorn(K, a.astype(np.float64), b.astype(np.float64), 200)
    plan2 = tfi.Plan.from_spec(t, delta, W.KernelSpec.powexp(1.0 / eps), leaf_max=256, max_channels=8)
    cost_gpu = np.einsum("ic,ic->c", u.double().cpu().numpy(), plan2.apply(v).double().cpu().numpy())
    cost_ref = S.transport_cost(S.dense_matrix(t, delta, W.KernelSpec.powexp(1.0 / eps)), uo, vo)
    assert np.all(np.abs(cost_gpu - cost_ref) <= 1e-3 * np.abs(cost_ref))
    ku = plan.apply(u).double().cpu().numpy()
    assert np.abs(v.double().cpu().numpy() * ku - b).max() <= 1e-4 * np.abs(b).max()


def test_sinkhorn_update_rule_short_trajectory():
    t, delta, spec, a, b, plan = _setup(0.5)
    u, v = plan.sinkhorn(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), iters=10)
    uo, vo = S.sinkhorn(S.dense_matrix(t, delta, spec), a.astype(np.float64), b.astype(np.float64), 10)
    for got, ref in ((u, uo), (v, vo)):
        g = got.double().cpu().numpy()
        assert (np.abs(g - ref).max(0) / np.abs(ref).max(0)).max() <= 1e-3


def test_apply_at_configured_eps_005_normwise():
    # the torus-MST operator at eps = 0.05, Delta = 1/256 on Dirichlet fields: one apply within the
    # FP32 normwise bound (most kernel samples underflow to zero in FP32)
    cfg = W.configs.torus_sinkhorn(n=3000, pairs=8)
    t, delta = cfg["tree"], cfg["delta"]
    spec = W.KernelSpec.exp(1.0 / 0.05)
    a, _ = W.dirichlet_pairs(t.n, 8, seed=1)
    plan = tfi.Plan.from_spec(t, delta, spec, leaf_max=256, max_channels=8)
    y = plan.apply(torch.from_numpy(a).cuda()).double().cpu().numpy()
    from oracle import brute
    ref = brute.integrate(t, delta, spec, a.astype(np.float64))
    assert (np.abs(y - ref).max(0) / np.abs(ref).max(0)).max() <= 1e-4


def test_sinkhorn_at_configured_eps_005_with_direct_tables_matches_fp64():
    # the torus-MST recipe at eps = 0.05, Delta = 1/256: 200 FP32 iterations with direct tables against
    # the FP64 dense iteration; transport cost with the x exp(-x / eps) kernel, also direct
    eps = 0.05
    cfg = W.configs.torus_sinkhorn(n=3000, pairs=8)
    t, delta, spec = cfg["tree"], cfg["delta"], cfg["kernel"]
    a, b = W.dirichlet_pairs(t.n, 8, seed=1)
    plan = tfi.Plan.from_spec(t, delta, spec, leaf_max=256, max_channels=8, direct_all=True)
    assert plan.info()["n_jobs_fft"] == 0 and plan.info()["trunc_len"] >= 0
    u, v = plan.sinkhorn(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), iters=200)
    uo, vo = S.sinkhorn(S.dense_matrix(t, delta, spec), a.astype(np.float64), b.astype(np.float64), 200)
    f2 = W.KernelSpec.powexp(1.0 / eps)
    plan2 = tfi.Plan.from_spec(t, delta, f2, leaf_max=256, max_channels=8, direct_all=True)
    cost_gpu = np.einsum("ic,ic->c", u.double().cpu().numpy(), plan2.apply(v).double().cpu().numpy())
    cost_ref = S.transport_cost(S.dense_matrix(t, delta, f2), uo, vo)
    assert np.all(np.abs(cost_gpu - cost_ref) <= 1e-4 * np.abs(cost_ref))
