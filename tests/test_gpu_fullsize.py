"""Full-size workloads on the GPU, checked on sampled outputs against the CPU oracle.

* 2,097,152 points on the (1, 0.5, 0.25) ellipsoid, kappa = 200: eps = 1e-4 (mixed, complex64)
  and eps = 1e-8 (mixed policy: double-float and float64 far-field levels, double-float near
  field, complex128);
* 524,288 points in the unit cube, kappa = 40, 64 right-hand sides, eps = 1e-5 (tensor-core
  near field);
* 32 uneven problems (N log-uniform in [8192, 131072], kappa uniform in [10, 60], 4 RHS,
  eps = 1e-5) in one graph launch;
* 131,072 sources on the unit sphere, 131,072 targets on the radius-1.5 sphere, kappa = 32,
  eps = 1e-6, loss sum |phi - phi*|^2 with phi* from charges perturbed by 1% N(0,1):
  source-position gradient (float32 positions) against the direct-sum gradient on 64
  sampled sources (float64 and mixed policies), central differences (step 1e-4, float64
  path) on 64 random coordinates, and the charge gradient (adjoint apply, complex64)
  against the direct-sum adjoint on 256 sampled sources.
"""
import numpy as np
import pytest

from oracle import direct
from paper_0911_4114_gb300 import FmmBatch, FmmPlan, workloads as wl
from gpu_util import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _apply(plan, q):
    import torch
    out = plan.apply(torch.as_tensor(q, device="cuda"))
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("eps,dtype", [(1e-4, np.complex64), (1e-8, np.complex128)])
def test_ellipsoid_2m(eps, dtype):
    """One buffer box (default) and the tuned plan shape (buffer = 0, the benchmark's plan)."""
    s, t = wl.points("ellipsoid2m")
    q = wl.charges(len(s), 0, wl.rng(2, salt=1)).astype(dtype)
    idx = np.sort(wl.rng(2, salt=2).choice(len(t), 500, replace=False))
    want = direct.direct(s, t[idx], q.astype(np.complex128), 200.0, block=8)
    for buffer in (1, 0):
        plan = FmmPlan(s, t, 200.0, eps, precision="mixed", buffer=buffer)
        got = _apply(plan, q)
        assert rel(got[idx], want) <= eps, buffer
        del plan


def test_cube_512k_64_rhs():
    """One buffer box (a float64 level 2) and the tuned plan shape (two buffer boxes; the
    leaf level the cost model picks for 64 right-hand sides)."""
    s, t = wl.points("cube512k_rhs64")
    q = wl.charges(len(s), 64, wl.rng(3, salt=1)).astype(np.complex64)
    idx = np.sort(wl.rng(3, salt=2).choice(len(t), 100, replace=False))
    want = direct.direct(s, t[idx], q.astype(np.complex128), 40.0, block=16)
    for buffer in (1, 0):
        plan = FmmPlan(s, t, 40.0, 1e-5, precision="mixed", max_rhs=64, buffer=buffer)
        got = _apply(plan, q)
        assert rel(got[idx], want) <= 1e-5, buffer
        del plan


def test_batch_32_uneven_problems():
    import torch
    g = wl.rng(3, salt=3)
    sizes = np.exp(g.uniform(np.log(8192), np.log(131072), 32)).astype(int)
    kappas = g.uniform(10.0, 60.0, 32)
    pts = [wl.cube(int(n), g) for n in sizes]
    batch = FmmBatch([(x, x, k, 1e-5) for x, k in zip(pts, kappas)], precision="mixed", max_rhs=4, buffer=0)
    qs = [wl.charges(len(x), 4, g).astype(np.complex64) for x in pts]
    outs = batch.apply([torch.as_tensor(q, device="cuda") for q in qs])
    torch.cuda.synchronize()
    for p in range(32):
        idx = np.sort(g.choice(len(pts[p]), 100, replace=False))
        want = direct.direct(pts[p], pts[p][idx], qs[p].astype(np.complex128), kappas[p], block=32)
        assert rel(outs[p].cpu().numpy().astype(np.complex128)[idx], want) <= 1e-5, p


SPHERES_ROOT = (-1.6, -1.6, -1.6, 3.2)   # fixed root cube: finite differences keep the tree


def _spheres_problem():
    s, t = wl.points("spheres131k_grad")
    s = s.astype(np.float32).astype(np.float64)        # float32 source positions
    t = t.astype(np.float32).astype(np.float64)
    g = wl.rng(4, salt=1)
    q = wl.charges(len(s), 0, g).astype(np.complex64).astype(np.complex128)
    qstar = q + 0.01 * wl.charges(len(s), 0, g)        # charges perturbed by 1% N(0,1)
    return s, t, q, qstar, g


def test_gradient_two_spheres_131k_finite_differences():
    """Loss sum_i |phi_i - phi*_i|^2 on the two-sphere problem (kappa = 32, eps = 1e-6),
    phi* the apply of the perturbed charges; float64 path.  The position gradient is checked
    against the oracle's direct-sum gradient on 64 sampled sources and against central
    differences (step 1e-4, plans rebuilt at y +- h e) on 64 random coordinates, of which
    those whose point stays in its leaf box (the FMM with a fixed tree is smooth there) are
    compared; at least 32 must be."""
    import torch
    s, t, q, qstar, g = _spheres_problem()
    kw = dict(precision="fp64", root=SPHERES_ROOT)
    plan = FmmPlan(s, t, 32.0, 1e-6, **kw)
    phistar = _apply(plan, qstar)
    resid = _apply(plan, q) - phistar
    grad = plan.grad_sources(torch.as_tensor(q, device="cuda"),
                             torch.as_tensor(2.0 * resid, device="cuda")).cpu().numpy()
    idx = np.sort(g.choice(len(s), 64, replace=False))
    want = direct.direct_grad_sources(s[idx], t, q[idx], resid, 32.0)
    assert rel(grad[idx], want) <= 20e-6
    info = plan.info()
    perm0 = plan.debug_get("SRC_PERM")
    h = 1e-4
    checked = 0
    for j, c in zip(g.integers(0, len(s), 64), g.integers(0, 3, 64)):
        vals = []
        ok = True
        for sgn in (1.0, -1.0):
            sp = s.copy()
            sp[j, c] += sgn * h
            p2 = FmmPlan(sp, t, 32.0, 1e-6, **kw)
            ok &= np.array_equal(p2.debug_get("SRC_PERM"), perm0) and p2.info()["lf"] == info["lf"]
            vals.append(float(np.sum(np.abs(_apply(p2, q) - phistar) ** 2)))
            del p2
        if not ok:
            continue
        fd = (vals[0] - vals[1]) / (2 * h)
        assert fd == pytest.approx(grad[j, c], rel=1e-4, abs=1e-4 * np.max(np.abs(grad))), (j, c)
        checked += 1
    print(f"two-sphere finite differences: {checked} of 64 coordinates compared")
    assert checked >= 32


def test_gradient_two_spheres_131k_mixed_and_charges():
    """The same loss under the mixed policy (phi and phi* from the mixed apply).  The
    gradients are vector-Jacobian products with the cotangent g = 2 (phi - phi*): the
    position gradient is checked against the direct-sum gradient with that cotangent on 64
    sampled sources, the charge gradient (the adjoint apply A^H g, complex64) against the
    direct-sum adjoint on 256 sampled sources."""
    import torch
    s, t, q, qstar, g = _spheres_problem()
    plan = FmmPlan(s, t, 32.0, 1e-6, precision="mixed")
    q64 = torch.as_tensor(q.astype(np.complex64), device="cuda")
    phi = plan.apply(q64).cpu().numpy().astype(np.complex128)
    phistar = _apply(plan, qstar.astype(np.complex64))
    gvec = (2.0 * (phi - phistar)).astype(np.complex64)
    gres = torch.as_tensor(gvec, device="cuda")
    grad = plan.grad_sources(q64, gres).cpu().numpy()
    idx = np.sort(g.choice(len(s), 64, replace=False))
    want = direct.direct_grad_sources(s[idx], t, q[idx], gvec.astype(np.complex128) / 2.0, 32.0)
    assert rel(grad[idx], want) <= 20e-6
    gq = plan.apply_adjoint(gres).cpu().numpy().astype(np.complex128)
    jdx = np.sort(g.choice(len(s), 256, replace=False))
    want_q = direct.direct_adjoint(s[jdx], t, gvec.astype(np.complex128), 32.0)
    assert rel(gq[jdx], want_q) <= 1e-5
