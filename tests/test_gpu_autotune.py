"""The library autotuner (tfi_autotune): the chosen leaf cutoff and shared-memory FFT
tile come from the candidates, and the plan it returns (tuned on a subset of a
forest's trees, or the winning plan itself for a single tree) matches the FP64
oracle. Every FFT tile size is also checked for parity on its own."""
import numpy as np
import pytest

import workloads as W
from oracle import brute

from ._lib import tfi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _err(y, ref):
    y = np.asarray(y, dtype=np.float64).reshape(ref.shape[0], -1)
    return float((np.abs(y - ref).max(0) / np.maximum(np.abs(ref).max(0), 1e-300)).max())


def test_autotune_forest_on_a_subset():
    cfg = W.configs.uneven_batch(count=40, lo=16, hi=3000, d=16)
    t = cfg["tree"]
    plan, tuned = tfi.Plan.autotune(t, cfg["delta"], cfg["kernel"], 16, leaf_candidates=[16, 64, 256],
                                    sample_trees=10, reps=2)
    assert tuned["leaf_max"] in (16, 64, 256)
    assert tuned["fft_cta_points"] in (4096, 8192, 16384)
    assert tuned["ms_per_apply"] > 0
    F = W.normal_field(t.n, 16, seed=123)
    y = plan.apply(torch.from_numpy(F).cuda()).cpu().numpy()
    tgt = np.sort(np.random.default_rng(0).choice(t.n, 300, replace=False)).astype(np.int32)
    ref = brute.integrate(t, cfg["delta"], cfg["kernel"], F.astype(np.float64), targets=tgt)
    assert _err(y[tgt], ref) <= 1e-4


def test_autotune_single_tree_returns_the_winning_plan():
    cfg = W.configs.sweep(shape="rrt", n=4096, d=16)
    t = cfg["tree"]
    plan, tuned = tfi.Plan.autotune(t, cfg["delta"], cfg["kernel"], 16, leaf_candidates=[64, 256], reps=2)
    assert tuned["leaf_max"] in (64, 256)
    F = W.normal_field(t.n, 16, seed=7)
    y = plan.apply(torch.from_numpy(F).cuda()).cpu().numpy()
    assert _err(y, brute.integrate(t, cfg["delta"], cfg["kernel"], F.astype(np.float64))) <= 1e-4


@pytest.mark.parametrize("cta", [4096, 8192, 16384])
@pytest.mark.parametrize("d", [3, 16, 64])
def test_fft_tile_sizes(cta, d):
    cfg = W.configs.sweep(shape="rrt", n=4096, d=d)
    t = cfg["tree"]
    plan = tfi.Plan.from_spec(t, cfg["delta"], cfg["kernel"], leaf_max=256, max_channels=d, fft_cta_points=cta)
    assert plan.info()["n_jobs_fft"] > 0
    F = W.normal_field(t.n, d, seed=8)
    y = plan.apply(torch.from_numpy(F).cuda()).cpu().numpy()
    assert _err(y, brute.integrate(t, cfg["delta"], cfg["kernel"], F.astype(np.float64))) <= 1e-4


def test_autotune_rejects_bad_arguments():
    cfg = W.configs.rrt_n2000()
    with pytest.raises(tfi.TfiError):
        tfi.Plan.autotune(cfg["tree"], cfg["delta"], cfg["kernel"], 32, max_channels=16)
    with pytest.raises(tfi.TfiError):
        tfi.Plan.autotune(cfg["tree"], cfg["delta"], cfg["kernel"], 16, reps=0)
