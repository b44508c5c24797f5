"""Float32 near field on the 5th-generation tensor cores (tcgen05.mma kind::tf32, 3xTF32
split products, accumulators in tensor memory), used from 16 right-hand sides; and the
device watchdog that its bounded mbarrier waits report through hfmm_query.

With no far field (one box, or boxes below a wavelength) the apply is the near field alone:
it must match the float64 direct sum to float32 accuracy, apply and adjoint, with ragged
source tiles, several flushes of the accumulator, right-hand-side counts that are not a
multiple of the 64 per pass, coincident points, and distinct targets; and each column must
match the one-RHS scalar kernel.
"""
import ctypes

import numpy as np
import pytest

from oracle import direct
from paper_0911_4114_gb300 import FmmPlan, workloads as wl
from paper_0911_4114_gb300 import _native as nat
from gpu_util import rel, run_apply

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("nrhs", [16, 40, 70])
def test_tc5_near_field_one_box(nrhs):
    import torch
    g = wl.rng(150, salt=nrhs)
    x = wl.cube(1500, g)
    x[10] = x[3]                                  # a coincident pair: skipped
    q = wl.charges(len(x), nrhs, g)
    lib = FmmPlan(x, x, 25.0, 1e-5, precision="mixed", max_leaf=4096, max_rhs=nrhs)
    assert lib.info()["near_precision"] == "fp32" and lib.info()["lf"] < 2
    got = run_apply(lib, q)
    want = direct.direct(x, x, q, 25.0)
    assert rel(got, want) <= 1e-6
    for r in (0, nrhs - 1):
        assert rel(run_apply(lib, q[:, r]), got[:, r]) <= 1e-6
    w = wl.charges(len(x), nrhs, g)
    adj = lib.apply_adjoint(torch.as_tensor(w, device="cuda")).cpu().numpy()
    assert rel(adj, direct.direct_adjoint(x, x, w, 25.0)) <= 1e-6
    assert lib.info() is not None                 # no watchdog report


def test_tc5_near_field_many_boxes_distinct_targets():
    g = wl.rng(151)
    s = wl.sphere(3000, g)
    t = wl.sphere(2000, g, radius=1.2)
    q = wl.charges(len(s), 24, g)
    lib = FmmPlan(s, t, 4.0, 1e-5, precision="mixed", max_leaf=64, max_rhs=24)
    info = lib.info()
    assert info["lf"] < 2 and info["nbox"][-1] > 1
    got = run_apply(lib, q)
    assert rel(got, direct.direct(s, t, q, 4.0)) <= 1e-6


def test_tc5_with_far_field():
    """A plan with a far field and 32 right-hand sides: the whole apply within eps."""
    g = wl.rng(152)
    x = wl.cube(6000, g)
    q = wl.charges(len(x), 32, g)
    lib = FmmPlan(x, x, 40.0, 1e-5, precision="mixed", max_rhs=32, buffer=2, depth=4)
    assert lib.info()["lf"] >= 2
    got = run_apply(lib, q)
    idx = np.sort(g.choice(len(x), 200, replace=False))
    assert rel(got[idx], direct.direct(x, x[idx], q, 40.0)) <= 1e-5


def test_watchdog_reports_timeout_and_context_survives():
    """A kernel whose bounded wait runs out (an mbarrier nothing completes) sets the plan's
    watchdog flag: hfmm_query returns HFMM_ERR_TIMEOUT once, then the plan works again."""
    import torch
    L = nat.lib()
    g = wl.rng(153)
    x = wl.cube(500, g)
    q = wl.charges(len(x), 0, g)
    lib = FmmPlan(x, x, 5.0, 1e-6, precision="mixed", max_leaf=64)
    assert L.hfmm_debug_watchdog_probe(lib._h, None) == nat.OK
    torch.cuda.synchronize()
    inf = nat.Info()
    assert L.hfmm_query(lib._h, ctypes.byref(inf)) == nat.ERR_TIMEOUT
    assert b"watchdog" in L.hfmm_last_error()
    assert L.hfmm_query(lib._h, ctypes.byref(inf)) == nat.OK
    got = run_apply(lib, q)
    assert rel(got, direct.direct(x, x, q, 5.0)) <= 1e-6
