"""GPU position gradient and autograd through the C ABI.

Checked against the oracle's direct-sum gradient of the same loss, against central
finite differences of the library's own float64 apply (plans rebuilt at y +- h e with the
root cube held, coordinates whose box changes are skipped), and the autograd Function
against explicit adjoint / gradient calls.
"""
import numpy as np
import pytest

from oracle import direct
from paper_0911_4114_gb300 import FmmPlan, workloads as wl
from gpu_util import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _problem(n=2500, m=2000, seed=80):
    g = wl.rng(seed)
    s = wl.sphere(n, g)
    t = wl.sphere(m, g, radius=1.5)
    q = wl.charges(n, 0, g)
    qstar = q + 0.01 * wl.charges(n, 0, g)
    return s, t, q, qstar


ROOT = (-1.6, -1.6, -1.6, 3.2)
KAPPA, EPS = 8.0, 1e-6


def _phi(plan, q):
    import torch
    out = plan.apply(torch.as_tensor(q, device="cuda"))
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gradient_matches_direct_sum_gradient(precision):
    import torch
    s, t, q, qstar = _problem()
    plan = FmmPlan(s, t, KAPPA, EPS, precision=precision, root=ROOT, max_leaf=32)
    assert plan.info()["lf"] >= 2
    phistar = direct.direct(s, t, qstar, KAPPA)
    resid = _phi(plan, q) - phistar
    g = torch.as_tensor(2.0 * resid, device="cuda")
    grad = plan.grad_sources(torch.as_tensor(q, device="cuda"), g).cpu().numpy()
    want = direct.direct_grad_sources(s, t, q, direct.direct(s, t, q, KAPPA) - phistar, KAPPA)
    assert rel(grad, want) <= 20 * EPS


def test_gradient_matches_finite_differences():
    s, t, q, qstar = _problem(n=1500, m=1200, seed=81)
    import torch
    phistar = direct.direct(s, t, qstar, KAPPA)

    def loss(src):
        p = FmmPlan(src, t, KAPPA, EPS, precision="fp64", root=ROOT, max_leaf=32)
        return float(np.sum(np.abs(_phi(p, q) - phistar) ** 2)), p.debug_get("SRC_PERM")

    plan = FmmPlan(s, t, KAPPA, EPS, precision="fp64", root=ROOT, max_leaf=32)
    resid = _phi(plan, q) - phistar
    grad = plan.grad_sources(torch.as_tensor(q, device="cuda"),
                             torch.as_tensor(2.0 * resid, device="cuda")).cpu().numpy()
    perm0 = plan.debug_get("SRC_PERM")
    rng = np.random.default_rng(82)
    h = 1e-4
    checked = 0
    for j, c in zip(rng.integers(0, len(s), 24), rng.integers(0, 3, 24)):
        sp, sm = s.copy(), s.copy()
        sp[j, c] += h
        sm[j, c] -= h
        lp, pp = loss(sp)
        lm, pm = loss(sm)
        if not (np.array_equal(pp, perm0) and np.array_equal(pm, perm0)):
            continue                        # the point moved to another box: FMM not smooth there
        fd = (lp - lm) / (2 * h)
        assert fd == pytest.approx(grad[j, c], rel=2e-5, abs=2e-5 * np.max(np.abs(grad))), (j, c)
        checked += 1
    assert checked >= 16


def test_autograd_function():
    import torch
    from paper_0911_4114_gb300.autograd import fmm_apply
    s, t, q, qstar = _problem(n=1200, m=900, seed=83)
    plan = FmmPlan(s, t, KAPPA, EPS, precision="fp64", root=ROOT, max_leaf=32)
    qt = torch.as_tensor(q, device="cuda").requires_grad_(True)
    yt = torch.as_tensor(s, device="cuda").requires_grad_(True)
    target = torch.as_tensor(direct.direct(s, t, qstar, KAPPA), device="cuda")
    phi = fmm_apply(qt, yt, plan)
    loss = torch.sum(torch.abs(phi - target) ** 2)
    loss.backward()
    g = 2.0 * (phi.detach() - target)
    want_q = plan.apply_adjoint(g)
    want_y = plan.grad_sources(qt.detach(), g)
    torch.cuda.synchronize()
    # autograd forms g through abs() and pow (ulp-level differences from 2 (phi - phi*)),
    # which the float64 levels' round-off amplification turns into ~1e-12 relative
    assert torch.allclose(qt.grad, want_q, rtol=1e-9, atol=1e-9 * float(want_q.abs().max()))
    assert torch.allclose(yt.grad, want_y, rtol=1e-9, atol=1e-9 * float(want_y.abs().max()))
