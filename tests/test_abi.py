"""The C ABI: libtfi loads, exports every function include/tfi.h declares, and
rejects bad input with the documented status codes (host-only plans, no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W

from ._lib import tfi

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "tfi.h")


def test_exports_every_declared_function():
    text = open(HEADER).read()
    declared = set(re.findall(r"^(?:tfi_status|const char \*)\s*(tfi_\w+)\s*\(", text, re.M))
    assert {"tfi_plan", "tfi_apply", "tfi_apply_backward", "tfi_destroy"} <= declared
    lib = ctypes.CDLL(tfi.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(tfi.EXPORTED_SYMBOLS)


def _plan(n, u, v, w, **kw):
    kw.setdefault("host_only", True)
    return tfi.Plan(n, u, v, w, **kw)


def test_rejects_cycle_and_bad_vertices():
    with pytest.raises(tfi.TfiError) as e:
        _plan(3, [0, 1, 2], [1, 2, 0], [1.0, 1.0, 1.0])
    assert e.value.name in ("ARG", "NOT_TREE")
    with pytest.raises(tfi.TfiError) as e:
        _plan(4, [0, 1, 2], [1, 2, 0], [1.0, 1.0, 1.0])
    assert e.value.name == "NOT_TREE"
    with pytest.raises(tfi.TfiError) as e:
        _plan(3, [0, 1], [1, 3], [1.0, 1.0])
    assert e.value.name == "NOT_TREE"
    with pytest.raises(tfi.TfiError) as e:
        _plan(3, [0, 1], [1, 1], [1.0, 1.0])
    assert e.value.name == "NOT_TREE"


@pytest.mark.parametrize("bad", [0.0, -1.0, float("nan"), float("inf")])
def test_rejects_bad_weights(bad):
    with pytest.raises(tfi.TfiError) as e:
        _plan(3, [0, 1], [1, 2], [1.0, bad])
    assert e.value.name == "WEIGHT"


def test_rejects_bad_options():
    for kw in (dict(delta=0.0), dict(delta=-1.0), dict(leaf_max=0), dict(leaf_max=5000), dict(max_channels=0),
               dict(kernel=("expsum", [1.0])), dict(kernel=("gauss", [1.0, 2.0, 3.0]))):
        with pytest.raises(tfi.TfiError) as e:
            _plan(3, [0, 1], [1, 2], [1.0, 1.0], **kw)
        assert e.value.name == "ARG"


def test_grid_overflow_and_short_table():
    with pytest.raises(tfi.TfiError) as e:
        _plan(3, [0, 1], [1, 2], [1e9, 1.0], delta=1e-3)
    assert e.value.name == "GRID_OVERFLOW"
    with pytest.raises(tfi.TfiError) as e:
        _plan(4, [0, 1, 2], [1, 2, 3], [1.0, 1.0, 1.0], kernel=("table", []), table=[1.0, 0.5], leaf_max=4)
    assert e.value.name == "GRID_OVERFLOW"
    p = _plan(4, [0, 1, 2], [1, 2, 3], [1.0, 1.0, 1.0], kernel=("table", []), table=[1.0, 0.5, 0.25, 0.125],
              leaf_max=4)
    assert p.info()["n_leaves"] == 1


def test_forest_and_singletons_plan_on_host():
    p = _plan(5, [0, 3], [1, 4], [1.0, 2.0], leaf_max=1)
    info = p.info()
    assert info["n"] == 5 and info["n_leaves"] + info["n_calls"] >= 3


def test_host_only_plan_cannot_apply():
    p = _plan(3, [0, 1], [1, 2], [1.0, 1.0])
    code = tfi.lib().tfi_apply(p._h, ctypes.c_void_p(8), ctypes.c_void_p(16), 1, 0, None)
    assert code == 9  # TFI_ERR_NO_DEVICE


def test_destroy_null_is_ok():
    assert tfi.lib().tfi_destroy(None) == 0


def test_quantisation_matches_oracle_rounding():
    # q_e = max(1, round(w/delta)) with ties to even, identical to numpy.rint
    from oracle.kernels import quantise
    w = np.array([0.5, 1.5, 2.5, 0.49, 3.5000001, 0.01, 7.0])
    p = _plan(8, list(range(7)), list(range(1, 8)), w, delta=1.0, policy="diameter", leaf_max=1)
    calls = p.export("calls")
    assert calls[0, 6] == quantise(w, 1.0).sum()


def test_rejects_bad_fft_tile():
    t = W.path(10)
    with pytest.raises(tfi.TfiError) as e:
        tfi.Plan.from_spec(t, 1.0, W.KernelSpec.exp(0.1), host_only=True, fft_cta_points=1000)
    assert e.value.name == "ARG"
