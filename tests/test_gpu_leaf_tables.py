"""Plane-wave tables of a float64 leaf level (S2M / L2T and their transposes read plane
waves evaluated once at plan time instead of evaluating float64 sincos per use).

The table-driven apply must agree with the on-the-fly apply of the same plan (tables turned
off with leaf_table_bytes=0) to the float64 round-off of the quadrature sums, forward and
adjoint, one and several right-hand sides, with sources = targets (one shared table) and
with distinct target points (two tables), under the float64 policy and under the mixed
policy with a float64 leaf; and stay within eps of the direct sum.
"""
import numpy as np
import pytest

from oracle import direct, fmm as ofmm
from paper_0911_4114_gb300 import FmmPlan, workloads as wl
from gpu_util import fp64_round_est, rel, run_apply

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _cases():
    g = wl.rng(120)
    x = wl.cube(4000, g)
    yield "cube_mixed_fp64_leaf", x, x, 56.0, 1e-4, "mixed", dict(depth=3, root=(0, 0, 0, 1.0))
    yield "cube_fp64", x, x, 56.0, 1e-6, "fp64", dict(depth=3, root=(0, 0, 0, 1.0))
    s = wl.sphere(5000, g)
    t = wl.sphere(3000, g, radius=1.5)
    yield "two_spheres_fp64", s, t, 20.0, 1e-6, "fp64", dict(max_leaf=32)


CASES = {c[0]: c[1:] for c in _cases()}


@pytest.mark.parametrize("name", sorted(CASES))
def test_tables_match_on_the_fly(name):
    import torch
    s, t, kappa, eps, prec, kw = CASES[name]
    R = 3
    on = FmmPlan(s, t, kappa, eps, precision=prec, max_rhs=R, **kw)
    off = FmmPlan(s, t, kappa, eps, precision=prec, max_rhs=R, leaf_table_bytes=0, **kw)
    i_on, i_off = on.info(), off.info()
    assert i_on["levels"][i_on["lf"]]["precision"] == "fp64"
    assert i_on["leaf_tables"] and not i_off["leaf_tables"]
    npair = i_on["levels"][i_on["lf"]]["K"] // 2
    rows = len(s) + (0 if t is s else len(t))
    assert i_on["leaf_table_bytes"] == rows * npair * 16
    orc = ofmm.Plan(s, t, kappa, eps, precision=prec, **kw)
    tol = max(1e-13, 16.0 * fp64_round_est(orc))
    g = wl.rng(121)
    q = wl.charges(len(s), R, g)
    w = wl.charges(len(t), R, g)
    a_on, a_off = run_apply(on, q), run_apply(off, q)
    d = np.max(np.abs(a_on - a_off)) / np.max(np.abs(a_off))
    print(f"leaf-tables {name}: apply max|diff|/max = {d:.3e} (tol {tol:.1e})")
    assert d <= tol
    one = run_apply(on, q[:, 1])
    assert np.max(np.abs(one - a_on[:, 1])) <= tol * np.max(np.abs(a_on))
    wt = torch.as_tensor(w, device="cuda")
    h_on = on.apply_adjoint(wt).cpu().numpy()
    h_off = off.apply_adjoint(wt).cpu().numpy()
    d = np.max(np.abs(h_on - h_off)) / np.max(np.abs(h_off))
    print(f"leaf-tables {name}: adjoint max|diff|/max = {d:.3e}")
    assert d <= tol
    assert rel(a_on[:, 0], direct.direct(s, t, q[:, 0], kappa)) <= eps
    assert rel(h_on[:, 0], direct.direct_adjoint(s, t, w[:, 0], kappa)) <= eps
