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


def test_option_and_state_errors():
    """Options outside their ranges and calls a host-only plan cannot serve are refused
    with status codes; quadratures beyond the device transform lengths are refused before
    the transfer tables are built."""
    import time
    L = nat.lib()
    rng = np.random.default_rng(1)
    x = rng.random((40, 3))
    h = ctypes.c_void_p()

    def plan_status(**kw):
        opt = nat.Options()
        L.hfmm_default_options(ctypes.byref(opt))
        opt.device = -1
        for k, v in kw.items():
            if k == "alphas":
                for i in range(4):
                    opt.alpha_ladder[i] = v[i] if i < len(v) else 0.0
            else:
                setattr(opt, k, v)
        return L.hfmm_plan(x.ctypes.data, 40, x.ctypes.data, 40, 5.0, 1e-6, ctypes.byref(opt), ctypes.byref(h))

    assert plan_status() == nat.OK
    L.hfmm_destroy(h)
    for bad in (dict(max_rhs=0), dict(max_rhs=5000), dict(depth=21), dict(depth=-1), dict(eps_scale=0.0),
                dict(eps_scale=1.5), dict(precision=7), dict(max_leaf=0), dict(alphas=(0.3,)),
                dict(alphas=(1.2,)), dict(alphas=())):
        assert plan_status(**bad) == nat.ERR_ARG, bad
    nan_t = x.copy()
    nan_t[3, 0] = np.inf
    assert L.hfmm_plan(x.ctypes.data, 40, nan_t.ctypes.data, 40, 5.0, 1e-6, None, ctypes.byref(h)) == nat.ERR_ARG
    assert L.hfmm_query(None, None) == nat.ERR_ARG
    assert L.hfmm_destroy(None) == nat.OK
    p = FmmPlan(x, x, 5.0, 1e-6, device=-1)
    for call in (lambda: p.apply_adjoint_ptr(1, 1, 1, nat.C128), lambda: p.set_timing(True)):
        with pytest.raises(nat.HfmmError) as e:
            call()
        assert e.value.status == nat.ERR_STATE
    # a very high-frequency coarse level needs N_theta > 1024: refused quickly
    t0 = time.perf_counter()
    with pytest.raises(nat.HfmmError) as e:
        FmmPlan(x, x, 4000.0, 1e-6, depth=2, root=(0, 0, 0, 1.0), device=-1)
    assert e.value.status == nat.ERR_ARG and b"above 1024" in L.hfmm_last_error()
    assert time.perf_counter() - t0 < 30.0


def test_require_far_flag_returns_unstable():
    """HFMM_FLAG_REQUIRE_FAR: a plan with no far-field level (boxes below a wavelength, or
    too few points for two levels) fails with HFMM_ERR_UNSTABLE and a reason; a plan with a
    far field is unaffected; without the flag the same inputs plan a pure near field."""
    L = nat.lib()
    rng = np.random.default_rng(2)
    x = rng.random((3000, 3))
    h = ctypes.c_void_p()

    def status(kappa, flags, **kw):
        opt = nat.Options()
        L.hfmm_default_options(ctypes.byref(opt))
        opt.device = -1
        opt.flags = flags
        for k, v in kw.items():
            setattr(opt, k, v)
        st = L.hfmm_plan(x.ctypes.data, len(x), x.ctypes.data, len(x), kappa, 1e-6, ctypes.byref(opt),
                         ctypes.byref(h))
        if st == nat.OK:
            L.hfmm_destroy(h)
        return st

    assert status(5.0, 0, max_leaf=16) == nat.OK                       # near field only, allowed
    assert status(5.0, nat.FLAG_REQUIRE_FAR, max_leaf=16) == nat.ERR_UNSTABLE
    assert b"wavelength" in L.hfmm_last_error()
    assert status(60.0, nat.FLAG_REQUIRE_FAR, max_leaf=16) == nat.OK    # kappa a_2 = 15
    assert status(60.0, nat.FLAG_REQUIRE_FAR, max_leaf=4000) == nat.ERR_UNSTABLE   # depth 0
    assert b"occupancy depth" in L.hfmm_last_error()
    assert status(60.0, 8, max_leaf=16) == nat.ERR_ARG                  # unknown flag bit
    assert status(60.0, 0, max_leaf=16, leaf_table_bytes=-2) == nat.ERR_ARG
    with pytest.raises(nat.HfmmError) as e:
        FmmPlan(x, x, 5.0, 1e-6, max_leaf=16, device=-1, require_far=True)
    assert e.value.status == nat.ERR_UNSTABLE


def test_host_allocation_failure_returns_nomem():
    """A host allocation failure at any planning stage (simulated by the planner's test hook)
    makes hfmm_plan return HFMM_ERR_NOMEM with a message and no plan; the hook is off afterwards
    and the same plan then succeeds."""
    L = nat.lib()
    x = np.random.default_rng(3).random((2500, 3))
    h = ctypes.c_void_p()

    def plan():
        opt = nat.Options()
        L.hfmm_default_options(ctypes.byref(opt))
        opt.device = -1
        opt.precision = nat.PREC_MIXED
        return L.hfmm_plan(x.ctypes.data, len(x), x.ctypes.data, len(x), 60.0, 1e-5, ctypes.byref(opt),
                           ctypes.byref(h))

    failed = 0
    for after in range(12):
        assert L.hfmm_debug_fail_host_alloc(after) == nat.OK
        st = plan()
        L.hfmm_debug_fail_host_alloc(-1)
        if st == nat.ERR_NOMEM:
            failed += 1
            assert b"allocation" in L.hfmm_last_error()
            assert not h.value
        else:
            assert st == nat.OK
            L.hfmm_destroy(h)
            break
    assert failed >= 5            # bounding cube, occupancy, levels, tree, at least one table
    assert plan() == nat.OK       # unaffected once the hook has fired
    L.hfmm_destroy(h)
