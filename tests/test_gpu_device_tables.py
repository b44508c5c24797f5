"""T^{s,LL} transfer tables computed on the device (Algorithm BMTF and the per-row
anterpolation of Section 3.3.2 as CUDA kernels, float64) against the host planner's tables
and against the oracle's directly computed tables, for one and two buffer boxes and every
storage precision; and the apply with device tables against the apply with host tables.
"""
import numpy as np
import pytest

from oracle import fmm as ofmm
from oracle import quadrature as oq
from paper_0911_4114_gb300 import FmmPlan, workloads as wl
from gpu_util import fp64_parity_tol, run_apply

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


CASES = [
    ("cube_b1", 60.0, 1e-6, dict(depth=3, root=(0, 0, 0, 1.0))),
    ("cube_b2", 70.0, 1e-6, dict(depth=3, root=(0, 0, 0, 1.0), buffer=2)),
]


@pytest.mark.parametrize("name,kappa,eps,kw", CASES, ids=[c[0] for c in CASES])
def test_device_tables_match_host_and_oracle(name, kappa, eps, kw):
    x = wl.cube(2500, wl.rng(140))
    host = FmmPlan(x, x, kappa, eps, precision="fp64", device=-1, **kw)
    dev = FmmPlan(x, x, kappa, eps, precision="fp64", **kw)
    orc = ofmm.Plan(x, x, kappa, eps, precision="fp64", **kw)
    assert dev.info()["lf"] == host.info()["lf"] == orc.lf >= 2
    for l in range(2, orc.lf + 1):
        vs = sorted(set(np.concatenate(list(orc.tree.vlist[l])).tolist()))
        est = orc.levels[l].rounding_estimate(oq.U_FP64)
        for v in vs[:: max(1, len(vs) // 16)]:
            a, b = dev.debug_get("TABLE", l, v), host.debug_get("TABLE", l, v)
            c = orc.table(l, v)
            scale = np.max(np.abs(c))
            # two float64 evaluations of the same steps in different orders (sums of many
            # terms of both signs): measured up to 8e-13 of max |T|
            assert np.max(np.abs(a - b)) <= 1e-11 * scale, (name, l, v)
            assert np.max(np.abs(a - c)) <= max(1e-11, 1e3 * est) * scale, (name, l, v)


def test_device_table_storage_precisions_and_apply():
    """Mixed policy (float32 and double-float levels store their tables in their own type):
    the stored tables equal the host's float64 tables rounded to that type (float32: 2e-7;
    double-float and float64: the 1e-11 agreement of two float64 evaluations); the float64 and mixed
    applies with device tables agree with those with host tables to round-off."""
    g = wl.rng(141)
    x = wl.cube(4000, g)
    kw = dict(depth=3, root=(0, 0, 0, 1.0))
    kappa = 56.0
    for prec, eps in (("mixed", 1e-4), ("mixed", 1e-9), ("fp64", 1e-6)):
        dev = FmmPlan(x, x, kappa, eps, precision=prec, **kw)
        hst = FmmPlan(x, x, kappa, eps, precision=prec, host_tables=True, **kw)
        ref = FmmPlan(x, x, kappa, eps, precision=prec, device=-1, **kw)
        info = dev.info()
        for l, lev in info["levels"].items():
            tol = {"fp32": 2e-7, "df": 1e-11, "fp64": 1e-11}[lev["precision"]]
            v = int(ref.debug_get("ILIST_V", l)[0])
            a, b = dev.debug_get("TABLE", l, v), ref.debug_get("TABLE", l, v)
            assert np.max(np.abs(a - b)) <= tol * np.max(np.abs(b)), (prec, eps, l)
        q = wl.charges(len(x), 0, g)
        got, want = run_apply(dev, q), run_apply(hst, q)
        orc = ofmm.Plan(x, x, kappa, eps, precision=prec, **kw)
        # float64: two sets of tables that agree to round-off give applies that agree to the
        # float64 parity bound (the quadrature sums amplify the table differences)
        tol = fp64_parity_tol(orc) if prec == "fp64" else eps / 10
        assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want)), (prec, eps)
