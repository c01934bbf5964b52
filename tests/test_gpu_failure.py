"""Failure detection on the device without a fault: the bounded mbarrier wait that
every tensor-core kernel uses gives up after its poll limit, records the failure
in a plan-owned flag and returns, leaving the context usable. The wait is made
to run out on a barrier that nothing arrives on (no MMA in flight, no tensor
memory held); the same call with an arrival completes."""
import numpy as np
import pytest

import workloads as W
from oracle import brute

from ._lib import tfi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    cfg = W.configs.rrt_n2000()
    t, d = cfg["tree"], 8
    plan = tfi.Plan.from_spec(t, cfg["delta"], cfg["kernel"], leaf_max=64, max_channels=d)
    assert plan.info()["device_errors"] == 0
    # an arrival completes the phase: the wait succeeds and no flag is set
    assert plan.selftest_wait(arrive=True, max_polls=10_000)
    assert plan.info()["device_errors"] == 0
    # nothing arrives: the wait runs out, the call reports TFI_ERR_TIMEOUT, the flag is counted
    assert not plan.selftest_wait(arrive=False, max_polls=10_000)
    assert plan.info()["device_errors"] == 1
    # the context is still usable: an apply after the timeout matches the oracle
    x = torch.from_numpy(W.normal_field(t.n, d, seed=5)).cuda()
    y = plan.apply(x).double().cpu().numpy()
    ref = brute.integrate(t, cfg["delta"], cfg["kernel"], x.double().cpu().numpy())
    assert float((np.abs(y - ref).max(0) / np.abs(ref).max(0)).max()) <= 1e-4
    # the next successful self-test clears the self-test's flag
    assert plan.selftest_wait(arrive=True, max_polls=100)
    assert plan.info()["device_errors"] == 0


def test_bounded_wait_rejects_bad_limits():
    cfg = W.configs.rrt_n2000()
    plan = tfi.Plan.from_spec(cfg["tree"], cfg["delta"], cfg["kernel"], leaf_max=64, max_channels=4)
    for bad in (0, -1, (1 << 26) + 1):
        with pytest.raises(tfi.TfiError) as e:
            plan.selftest_wait(arrive=False, max_polls=bad)
        assert e.value.name == "ARG"
