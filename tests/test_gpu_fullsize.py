"""Full-size workloads on the GPU, checked on sampled outputs against the CPU oracle.

* 2,097,152 points on the (1, 0.5, 0.25) ellipsoid, kappa = 200: eps = 1e-4 (mixed, complex64)
  and eps = 1e-8 (mixed policy: double-float and float64 far-field levels, double-float near
  field, complex128);
* 524,288 points in the unit cube, kappa = 40, 64 right-hand sides, eps = 1e-5 (tensor-core
  near field);
* 32 uneven problems (N log-uniform in [8192, 131072], kappa uniform in [10, 60], 4 RHS,
  eps = 1e-5) in one graph launch;
* 131,072 sources on the unit sphere, 131,072 targets on the radius-1.5 sphere, kappa = 32,
  eps = 1e-6: source-position gradient (float32 positions) against the direct-sum
  vector-Jacobian product on 64 sampled sources, and central differences (step 1e-4,
  float64 path) on 8 sampled coordinates.
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
    s, t = wl.points("ellipsoid2m")
    q = wl.charges(len(s), 0, wl.rng(2, salt=1)).astype(dtype)
    plan = FmmPlan(s, t, 200.0, eps, precision="mixed")
    got = _apply(plan, q)
    idx = np.sort(wl.rng(2, salt=2).choice(len(t), 500, replace=False))
    want = direct.direct(s, t[idx], q.astype(np.complex128), 200.0, block=8)
    assert rel(got[idx], want) <= eps


def test_cube_512k_64_rhs():
    s, t = wl.points("cube512k_rhs64")
    q = wl.charges(len(s), 64, wl.rng(3, salt=1)).astype(np.complex64)
    plan = FmmPlan(s, t, 40.0, 1e-5, precision="mixed", max_rhs=64)
    got = _apply(plan, q)
    idx = np.sort(wl.rng(3, salt=2).choice(len(t), 100, replace=False))
    want = direct.direct(s, t[idx], q.astype(np.complex128), 40.0, block=16)
    assert rel(got[idx], want) <= 1e-5


def test_batch_32_uneven_problems():
    import torch
    g = wl.rng(3, salt=3)
    sizes = np.exp(g.uniform(np.log(8192), np.log(131072), 32)).astype(int)
    kappas = g.uniform(10.0, 60.0, 32)
    pts = [wl.cube(int(n), g) for n in sizes]
    batch = FmmBatch([(x, x, k, 1e-5) for x, k in zip(pts, kappas)], precision="mixed", max_rhs=4)
    qs = [wl.charges(len(x), 4, g).astype(np.complex64) for x in pts]
    outs = batch.apply([torch.as_tensor(q, device="cuda") for q in qs])
    torch.cuda.synchronize()
    for p in range(0, 32, 4):
        idx = np.sort(g.choice(len(pts[p]), 100, replace=False))
        want = direct.direct(pts[p], pts[p][idx], qs[p].astype(np.complex128), kappas[p], block=32)
        assert rel(outs[p].cpu().numpy().astype(np.complex128)[idx], want) <= 1e-5, p


def test_gradient_two_spheres_131k():
    import torch
    s, t = wl.points("spheres131k_grad")
    s = s.astype(np.float32).astype(np.float64)        # float32 source positions
    t = t.astype(np.float32).astype(np.float64)
    g = wl.rng(4, salt=1)
    q = wl.charges(len(s), 0, g)
    w = wl.charges(len(t), 0, g)                       # any cotangent: the gradient is a VJP
    plan = FmmPlan(s, t, 32.0, 1e-6, precision="fp64")
    grad = plan.grad_sources(torch.as_tensor(q, device="cuda"), torch.as_tensor(w, device="cuda")).cpu().numpy()
    idx = np.sort(g.choice(len(s), 64, replace=False))
    want = direct.direct_grad_sources(s[idx], t, q[idx], w / 2.0, 32.0)
    assert rel(grad[idx], want) <= 20e-6
    # central differences of the library's own loss on a few coordinates
    qstar = q + 0.01 * wl.charges(len(s), 0, g)
    phistar = _apply(plan, qstar)
    resid = _apply(plan, q) - phistar
    g2 = plan.grad_sources(torch.as_tensor(q, device="cuda"), torch.as_tensor(2.0 * resid, device="cuda")).cpu().numpy()
    info = plan.info()
    perm0 = plan.debug_get("SRC_PERM")
    h = 1e-4
    checked = 0
    for j, c in zip(g.integers(0, len(s), 8), g.integers(0, 3, 8)):
        vals = []
        ok = True
        for sgn in (1.0, -1.0):
            sp = s.copy()
            sp[j, c] += sgn * h
            p2 = FmmPlan(sp, t, 32.0, 1e-6, precision="fp64")
            ok &= np.array_equal(p2.debug_get("SRC_PERM"), perm0) and p2.info()["lf"] == info["lf"]
            vals.append(float(np.sum(np.abs(_apply(p2, q) - phistar) ** 2)))
        if not ok:
            continue
        fd = (vals[0] - vals[1]) / (2 * h)
        assert fd == pytest.approx(g2[j, c], rel=1e-4, abs=1e-4 * np.max(np.abs(g2))), (j, c)
        checked += 1
    assert checked >= 4
