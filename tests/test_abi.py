"""The C-ABI library loads, exports every entry point declared in include/hfmm.h, and
rejects bad arguments with status codes (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_0911_4114_gb300 import FmmPlan
from paper_0911_4114_gb300 import _native as nat

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "hfmm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hfmm_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    L = nat.lib()
    names = declared_functions()
    assert "hfmm_plan" in names and "hfmm_apply" in names
    for name in names:
        assert hasattr(L, name), name
    assert set(nat.EXPORTS) <= set(names)


def test_bad_arguments():
    L = nat.lib()
    x = np.zeros((4, 3))
    h = ctypes.c_void_p()
    assert L.hfmm_plan(x.ctypes.data, 0, x.ctypes.data, 4, 1.0, 1e-6, None, ctypes.byref(h)) == nat.ERR_ARG
    assert L.hfmm_plan(x.ctypes.data, 4, x.ctypes.data, 4, -1.0, 1e-6, None, ctypes.byref(h)) == nat.ERR_ARG
    assert L.hfmm_plan(x.ctypes.data, 4, x.ctypes.data, 4, 1.0, 0.5, None, ctypes.byref(h)) == nat.ERR_ARG
    bad = x.copy()
    bad[1, 2] = np.nan
    assert L.hfmm_plan(bad.ctypes.data, 4, x.ctypes.data, 4, 1.0, 1e-6, None, ctypes.byref(h)) == nat.ERR_ARG
    assert b"finite" in L.hfmm_last_error()
    with pytest.raises(nat.HfmmError):
        FmmPlan(x, x, 1.0, 1e-6, root=(0.5, 0.5, 0.5, 0.1), device=-1)   # points outside the root cube


def test_host_only_plan_refuses_apply():
    rng = np.random.default_rng(0)
    x = rng.random((50, 3))
    p = FmmPlan(x, x, 3.0, 1e-6, device=-1)
    with pytest.raises(nat.HfmmError) as e:
        p.apply_ptr(1, 1, 1, nat.C128)
    assert e.value.status == nat.ERR_STATE
    info = p.info()
    assert info["lf"] <= 1 and info["p2p_pairs"] == 50 * 50


def test_degenerate_inputs_plan():
    x = np.array([[0.5, 0.5, 0.5]])
    p = FmmPlan(x, x, 1.0, 1e-6, device=-1)
    assert p.info()["p2p_pairs"] == 1
    y = np.repeat(x, 10, axis=0)           # coincident points
    p = FmmPlan(y, y, 1.0, 1e-6, max_leaf=4, device=-1)
    assert p.info()["lf"] <= 1
