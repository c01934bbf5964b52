"""Sinkhorn on the tree metric (Eq. app-sinkhorn-updates): the device driver
(FP32, graph-replayed iterations) against the FP64 dense oracle, on the
torus-MST workload recipe at a size the dense oracle handles."""
import numpy as np
import pytest

import workloads as W
from oracle import sinkhorn as S

from ._lib import tfi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_sinkhorn_torus_mst_matches_fp64_oracle():
    cfg = W.configs.torus_sinkhorn(n=3000, pairs=8)
    t, delta, eps = cfg["tree"], cfg["delta"], 0.05
    a, b = W.dirichlet_pairs(t.n, 8, seed=1)
    plan = tfi.Plan.from_spec(t, delta, cfg["kernel"], leaf_max=256, max_channels=8)
    u, v = plan.sinkhorn(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), iters=200)
    K = S.dense_matrix(t, delta, cfg["kernel"])
    uo, vo = S.sinkhorn(K, a.astype(np.float64), b.astype(np.float64), 200)
    # transport cost of diag(u) K diag(v): GPU applies K2 = x exp(-x/eps) with its own plan
    plan2 = tfi.Plan.from_spec(t, delta, W.KernelSpec.powexp(1.0 / eps), leaf_max=256, max_channels=8)
    k2v = plan2.apply(v).double().cpu().numpy()
    cost_gpu = np.einsum("ic,ic->c", u.double().cpu().numpy(), k2v)
    K2 = S.dense_matrix(t, delta, W.KernelSpec.powexp(1.0 / eps))
    cost_ref = S.transport_cost(K2, uo, vo)
    assert np.all(np.abs(cost_gpu - cost_ref) <= 1e-3 * np.abs(cost_ref))
    # the marginal constraint after the v update holds for the device scalings too
    ku = plan.apply(u).double().cpu().numpy()
    assert np.abs(v.double().cpu().numpy() * ku - b).max() <= 1e-4 * np.abs(b).max()
