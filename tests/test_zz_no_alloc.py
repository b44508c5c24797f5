"""hfmm_direct_noalloc: the near-field sum for callers that cannot allocate device memory.

Such callers (code inside a host framework's operator that may only use the framework's
memory pool, or code on a latency-critical path where an allocation would synchronise
streams) cannot create a plan, because planning allocates.  The entry point takes device
inputs and outputs and keeps its scratch in a fixed static device array.  It must agree
with the planned apply, which for a plan whose whole tree is one box is the same
mixed-precision direct sum, on two calls in a row (the second reuses the array the first
one filled).  This file is collected last so a stop-at-first-failure run has already run
every other test.
"""
import ctypes

import numpy as np
import pytest

from oracle import direct
from paper_0911_4114_gb300 import FmmPlan, workloads as wl
from paper_0911_4114_gb300 import _native as nat
from paper_0911_4114_gb300.plan import direct_noalloc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _planned(s, t, q, kappa):
    import torch
    plan = FmmPlan(s, t, kappa, 1e-6, precision="mixed", max_leaf=len(s) + len(t), max_rhs=q.shape[1])
    assert plan.info()["lf"] <= 1          # one box: the planned near field is the direct sum
    out = plan.apply(torch.as_tensor(q, device="cuda"))
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.complex128)


def _noalloc(s, t, q, kappa):
    import torch
    out = direct_noalloc(torch.as_tensor(s, device="cuda"), torch.as_tensor(t, device="cuda"),
                         torch.as_tensor(q, device="cuda"), kappa)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.complex128)


def test_two_calls_match_planned_apply():
    g = wl.rng(40)
    cases = [
        (wl.sphere(3000, g), wl.sphere(2000, g, radius=1.5), 2, np.complex128, 12.0),
        (wl.cube(1500, g) * 0.3 + 2.0, None, 1, np.complex64, 30.0),   # smaller, shifted box
    ]
    for s, t, r, dt, kappa in cases:
        if t is None:
            t = s
        q = wl.charges(len(s), r, g).astype(dt)
        got = _noalloc(s, t, q, kappa)
        want = _planned(s, t, q, kappa)
        assert np.linalg.norm(got - want) <= 1e-6 * np.linalg.norm(want)
        exact = direct.direct(s, t, q.astype(np.complex128), kappa)
        assert np.linalg.norm(got - exact) <= 1e-6 * np.linalg.norm(exact)


def test_rejects_sizes_above_the_static_limit():
    L = nat.lib()
    n = nat.NOALLOC_MAX_POINTS // 2 + 1
    st = L.hfmm_direct_noalloc(ctypes.c_void_p(8), n, ctypes.c_void_p(8), n, ctypes.c_void_p(8),
                               ctypes.c_void_p(8), 1, nat.C64, 1.0, None)
    assert st == nat.ERR_ARG
    assert b"static scratch limit" in L.hfmm_last_error()
