"""GPU adjoint apply (transposed FMM) through the C ABI.

Dot-product identity <A x, y> = <x, A^H y> with the library's own forward apply (the
transposition is exact up to round-off: bound from the plan's round-off estimate, floor
1e-12, float64 path), and A^H y against the oracle's direct-sum adjoint within eps.
"""
import numpy as np
import pytest

from oracle import direct, fmm as ofmm
from paper_0911_4114_gb300 import FmmPlan, workloads as wl
from gpu_util import fp64_parity_tol, fp64_round_est, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _cases():
    g = wl.rng(70)
    yield "cube_hf", wl.cube(2500, g), None, 60.0, 1e-6, dict(depth=3, root=(0, 0, 0, 1.0))
    s = wl.sphere(3000, g)
    t = wl.sphere(2000, g, radius=1.5)
    yield "two_spheres", s, t, 12.0, 1e-6, dict(max_leaf=16)
    x = wl.sphere(6000, g)
    yield "sphere", x, None, 24.0, 1e-6, dict(max_leaf=32)


CASES = {c[0]: c[1:] for c in _cases()}


def _run(plan, fn, v, dtype):
    import torch
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    out = getattr(plan, fn)(torch.as_tensor(np.ascontiguousarray(v)).to(device="cuda", dtype=tdt))
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_dot_product_identity_and_direct_adjoint(name, precision):
    s, t, kappa, eps, kw = CASES[name]
    t = s if t is None else t
    g = wl.rng(71)
    x = wl.charges(len(s), 2, g)
    y = wl.charges(len(t), 2, g)
    plan = FmmPlan(s, t, kappa, eps, precision=precision, max_rhs=2, **kw)
    dt = "c128"
    ax = _run(plan, "apply", x, dt)
    ahy = _run(plan, "apply_adjoint", y, dt)
    lhs = np.vdot(y, ax)          # <A x, y> = y^H A x
    rhs = np.vdot(ahy, x)         # <x, A^H y> = (A^H y)^H x
    scale = np.linalg.norm(ax) * np.linalg.norm(y)
    if precision == "fp64":
        orc = ofmm.Plan(s, t, kappa, eps, precision="fp64", **kw)
        tol = fp64_parity_tol(orc)
        print(f"fp64-dot {name}: |<Ax,y> - <x,A^H y>|/(|Ax||y|) = {abs(lhs - rhs) / scale:.3e}  "
              f"est = {fp64_round_est(orc):.3e}")
    else:
        tol = 1e-6
    assert abs(lhs - rhs) <= tol * scale, (name, abs(lhs - rhs) / scale)
    assert rel(ahy, direct.direct_adjoint(s, t, y, kappa)) <= eps


def test_adjoint_single_rhs_and_c64():
    s, t, kappa, eps, kw = CASES["two_spheres"]
    y = wl.charges(len(t), 0, wl.rng(72)).astype(np.complex64)
    plan = FmmPlan(s, t, kappa, eps, precision="mixed", **kw)
    got = _run(plan, "apply_adjoint", y, "c64")
    assert got.shape == (len(s),)
    assert rel(got, direct.direct_adjoint(s, t, y.astype(np.complex128), kappa)) <= eps
