"""Dense tensor-core evaluation (tcgen05) of the same operator, against the
FP64 oracle: f(D) tiles generated on chip, BF16 hi/lo split operands, FP32
accumulation in tensor memory."""
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


def _tree(n, seed, lo=1, hi=4):
    rng = np.random.default_rng(seed)
    t = W.random_recursive(n, rng)
    return t.with_weights(W.trees.integer_weights(t.m, lo, hi, rng))


@pytest.mark.parametrize("n,d", [(1, 16), (5, 16), (130, 16), (300, 3), (700, 33)])
def test_dense_f32_small(n, d):
    t = _tree(n, n)
    spec = W.KernelSpec.exp(0.2)
    p = tfi.Plan.from_spec(t, 1.0, spec, leaf_max=64, max_channels=d)
    F = W.normal_field(n, d, seed=5)
    y = p.dense_apply(torch.from_numpy(F).cuda()).cpu().numpy()
    assert _err(y, brute.integrate(t, 1.0, spec, F.astype(np.float64))) <= 1e-4


def test_dense_bf16_attention_trees():
    cfg = W.configs.attention(heads=3)
    trees = [h["tree"] for h in cfg["heads"]]
    f, _ = W.forest(trees)
    spec = cfg["heads"][0]["kernel"]
    p = tfi.Plan.from_spec(f, 1.0, spec, leaf_max=256, max_channels=128)
    F = torch.from_numpy(W.normal_field(f.n, 128, seed=9)).cuda().to(torch.bfloat16)
    y = p.dense_apply(F).float().cpu().numpy()
    ref = brute.integrate(f, 1.0, spec, F.float().cpu().numpy().astype(np.float64))
    assert _err(y, ref) <= 1e-2


def test_dense_matches_stad_weighted_forest():
    cfg = W.configs.uneven_batch(count=12, lo=50, hi=900, d=16)
    t = cfg["tree"]
    p = tfi.Plan.from_spec(t, cfg["delta"], cfg["kernel"], leaf_max=64, max_channels=16)
    x = torch.from_numpy(W.normal_field(t.n, 16, seed=3)).cuda()
    yd = p.dense_apply(x).cpu().numpy()
    ys = p.apply(x).cpu().numpy()
    ref = brute.integrate(t, cfg["delta"], cfg["kernel"], x.cpu().numpy().astype(np.float64))
    assert _err(yd, ref) <= 1e-4 and _err(ys, ref) <= 1e-4
