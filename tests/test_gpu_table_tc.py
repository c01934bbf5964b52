"""GPU parity of the tensor-core direct tables (tcgen05 kind::tf32) against the
FP64 oracle and against the FP32-ALU direct kernel, through the C ABI.

For d > 16 (for d = 16 from 512 bins) a table evaluated by direct summation with
64 .. 4096 bins is an f(r_i + r_j + |x_i - x_j|) x S product on the tensor cores
(both operands split into TF32 hi + lo, a fresh accumulator per 32 source bins);
TFI_PLAN_TABLES_ALU keeps every table on the FP32 ALUs. The N = 4096 sweep trees
at s0 = 64 have such tables on all three shapes (component corrections and call
cross tables), the caterpillar up to 1991 bins; the 8192-vertex caterpillar has
tables of up to 4007 bins, and under the diameter policy with every table summed
directly one of 8135 bins, which stays on the ALU kernel. Tolerance 1e-4 per
channel, normwise, for FP32 fields; 1e-2 for BF16 fields.
"""
import numpy as np
import pytest

import workloads as W
from oracle import brute

from ._lib import tfi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-4, "bf16": 1e-2}


def _err(y, ref):
    y = np.asarray(y, dtype=np.float64).reshape(ref.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return float((np.abs(y - ref).max(0) / np.maximum(np.abs(ref).max(0), 1e-300)).max())


def _eligible(p, d=17):
    # direct tables the tensor cores take at d channels
    jobs = p.export("jobs")
    nb = jobs[:, 3]
    lo = 64 if d > 16 else 512 if d == 16 else 1 << 30
    return int(((jobs[:, 0] == 1) & (nb >= lo) & (nb <= 4096)).sum())


def _run(t, delta, spec, d, dtype="f32", seed=5, **kw):
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    F = torch.from_numpy(W.normal_field(t.n, d, seed=seed)).to("cuda", tdt)
    p = tfi.Plan.from_spec(t, delta, spec, max_channels=d, **kw)
    q = tfi.Plan.from_spec(t, delta, spec, max_channels=d, tables_alu=True, **kw)
    y, y2, yq = p.apply(F), p.apply(F), q.apply(F)
    torch.cuda.synchronize()
    assert p.info()["device_errors"] == 0
    assert torch.equal(y, y2)   # fixed summation order
    ref = brute.integrate(t, delta, spec, F.float().cpu().numpy().astype(np.float64))
    return p, y, yq, _err(y.float().cpu().numpy(), ref), _err(yq.float().cpu().numpy(), ref)


@pytest.mark.parametrize("shape", ["rrt", "binary", "caterpillar"])
@pytest.mark.parametrize("d", [17, 32, 33, 64, 100])
def test_tables_on_tensor_cores(shape, d):
    # channel blocks of 32 / 64 with ragged ends, odd d (scalar bin-sum loads)
    cfg = W.configs.sweep(shape=shape, n=4096, d=d, kernel="exp")
    p, y, yq, e, e_alu = _run(cfg["tree"], cfg["delta"], cfg["kernel"], d, leaf_max=64)
    assert _eligible(p) > 0
    assert not torch.equal(y, yq)   # the tensor-core tables ran (another summation order)
    assert e <= TOL["f32"] and e_alu <= TOL["f32"]


@pytest.mark.parametrize("kernel", ["cauchy", "gauss"])
def test_two_dimensional_and_large_tables(kernel):
    # every table summed directly under the diameter policy: two-dimensional call cross tables of
    # up to 2548 bins; the 8192-vertex caterpillar's tables of up to 4007 bins at d = 24 and d = 16,
    # and under the diameter policy one of 8135 bins (on the ALU kernel)
    cfg = W.configs.sweep(shape="rrt", n=4096, d=24, kernel=kernel)
    p, _, _, e, e_alu = _run(cfg["tree"], cfg["delta"], cfg["kernel"], 24, leaf_max=16, policy="diameter",
                             direct_all=True)
    assert _eligible(p) > 0 and p.export("jobs")[:, 3].max() > 2048
    assert e <= TOL["f32"] and e_alu <= TOL["f32"]
    cfg = W.configs.sweep(shape="caterpillar", n=8192, d=24, kernel=kernel)
    for d, kw in ((24, {}), (16, {}), (24, {"policy": "diameter", "direct_all": True})):
        p, y, yq, e, _ = _run(cfg["tree"], cfg["delta"], cfg["kernel"], d, leaf_max=64 if not kw else 16, **kw)
        assert e <= TOL["f32"]
        assert _eligible(p, d) == 0 or not torch.equal(y, yq)


def test_bf16_fields_and_positive_sums():
    # BF16 fields (their bin sums are FP32 too); a positive field with a fast-decaying kernel, where
    # every output is a sum of positive terms and keeps a small error relative to itself
    cfg = W.configs.sweep(shape="binary", n=4096, d=64, kernel="exp")
    _, _, _, e, e_alu = _run(cfg["tree"], cfg["delta"], cfg["kernel"], 64, dtype="bf16", leaf_max=64)
    assert e <= TOL["bf16"] and e_alu <= TOL["bf16"]
    cfg = W.configs.sweep(shape="rrt", n=4096, d=32, kernel="exp")
    t = cfg["tree"]
    F = torch.from_numpy(np.abs(W.normal_field(t.n, 32, seed=8)) + 0.01).cuda()
    spec = W.KernelSpec.exp(2.0)
    p = tfi.Plan.from_spec(t, cfg["delta"], spec, leaf_max=64, max_channels=32, direct_all=True)
    assert _eligible(p) > 0
    y = p.apply(F).double().cpu().numpy()
    ref = brute.integrate(t, cfg["delta"], spec, F.cpu().numpy().astype(np.float64))
    assert float((np.abs(y - ref) / ref).max()) <= 1e-5
