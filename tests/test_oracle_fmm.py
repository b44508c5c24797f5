"""Pins of the oracle FMM against the direct sum and the paper's multi-level claim."""
import numpy as np
import pytest

from oracle import direct, fmm
from oracle import quadrature as qd


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _charges(rng, n, r=1):
    return (rng.standard_normal((n, r)) + 1j * rng.standard_normal((n, r))).squeeze()


def test_small_cube_low_frequency():
    """Uniform cube, kappa = 8 pi, eps = 1e-6, depth 3 requested (low-frequency breakdown cuts it)."""
    rng = np.random.default_rng(20260000)
    x = rng.random((1500, 3))
    q = _charges(rng, 1500)
    p = fmm.Plan(x, x, 8 * np.pi, 1e-6, depth=3, root=(0, 0, 0, 1.0))
    assert p.lf == 2
    assert _rel(fmm.apply(p, q), direct.direct(x, x, q, 8 * np.pi)) < 1e-6


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cube_two_levels(precision):
    rng = np.random.default_rng(7)
    x = rng.random((1200, 3))
    q = _charges(rng, 1200)
    kappa = 60.0
    p = fmm.Plan(x, x, kappa, 1e-6, depth=3, root=(0, 0, 0, 1.0), precision=precision)
    assert p.lf == 3
    assert _rel(fmm.apply(p, q), direct.direct(x, x, q, kappa)) < 1e-6


def test_sources_differ_from_targets_multi_rhs():
    rng = np.random.default_rng(11)
    s = rng.standard_normal((700, 3))
    s /= np.linalg.norm(s, axis=1)[:, None]
    t = rng.standard_normal((500, 3))
    t *= 1.5 / np.linalg.norm(t, axis=1)[:, None]
    q = _charges(rng, 700, 3)
    kappa = 12.0
    p = fmm.Plan(s, t, kappa, 1e-6, max_leaf=16)
    assert p.lf >= 2
    phi = fmm.apply(p, q)
    assert _rel(phi, direct.direct(s, t, q, kappa)) < 1e-6
    # summation order differs between R = 3 and R = 1: agreement to the plan's round-off estimate
    tol = max(1e-13, 16 * max(lp.rounding_estimate(qd.U_FP64) for lp in p.levels.values()))
    for r in range(3):
        assert np.max(np.abs(fmm.apply(p, q[:, r]) - phi[:, r])) < tol * np.abs(phi).max()


def test_coincident_points_are_skipped():
    x = np.array([[0.1, 0.2, 0.3], [0.1, 0.2, 0.3], [0.6, 0.7, 0.8]])
    q = np.array([1.0, 2.0, 3.0j])
    phi = direct.direct(x, x, q, 5.0)
    r = np.linalg.norm(x[2] - x[0])
    g = np.exp(5j * r) / r
    assert np.allclose(phi, [3.0j * g, 3.0j * g, 3.0 * g])


def _chain_error(kappa, depth, eps_l, y, x):
    """Section 3.5.2 setting: two points in far-apart level-2 boxes (a_2 = 1), M2L at level 2,
    depth-2 extra translation levels above the leaf; returns the relative error."""
    side = 4.0
    corner = np.zeros(3)
    plans = {l: qd.LevelPlan(kappa, side / 2 ** l, eps_l, 0.8) for l in range(2, depth + 1)}

    def center(p, l):
        h = side / 2 ** l
        return corner + (np.floor(p / h) + 0.5) * h

    quad = plans[depth].quad
    m = np.exp(1j * kappa * (quad.shat @ (y - center(y, depth))))
    for l in range(depth, 2, -1):
        up = qd.requadrature(m, plans[l].quad, plans[l - 1].quad)
        m = up * np.exp(1j * kappa * (plans[l - 1].quad.shat @ (center(y, l) - center(y, l - 1))))
    t = qd.tsll(plans[2].ell, kappa, center(y, 2) - center(x, 2), plans[2].ntheta, plans[2].nphi)
    loc = t * m
    for l in range(2, depth):
        sh = loc * np.exp(1j * kappa * (plans[l].quad.shat @ (center(x, l) - center(x, l + 1))))
        loc = qd.requadrature(sh, plans[l].quad, plans[l + 1].quad)
    q = plans[depth].quad
    val = np.sum(q.w * loc * np.exp(1j * kappa * (q.shat @ (center(x, depth) - x))))
    d = np.linalg.norm(x - y)
    g = np.exp(1j * kappa * d) / d
    return abs(val - g) / abs(g)


@pytest.mark.parametrize("y,x,bound", [
    # opposite corners (Figure WorstCaseBox): |r| ~ sqrt(3) a, beyond the design radius
    ((0.02, 0.03, 0.01), (2.97, 0.98, 0.99), 1e-3),
    # |r| = 0.7 sqrt(3) a, inside the design radius alpha sqrt(3) a = 0.8 sqrt(3) a
    ((0.15, 0.15, 0.15), (2.85, 0.85, 0.85), 2e-7),
])
def test_multilevel_error_independent_of_depth(y, x, bound):
    """Section 3.5.2 / Figure Error_Quad: adding translation levels leaves the error unchanged."""
    errs = [_chain_error(20.0, depth, 1e-7, np.array(y), np.array(x)) for depth in (2, 3, 4)]
    assert errs[0] < bound
    assert max(errs) - min(errs) < 1e-10


def test_adjoint_and_gradient_direct():
    rng = np.random.default_rng(2)
    s = rng.random((40, 3))
    t = rng.random((30, 3)) + 0.5
    kappa = 7.0
    q = _charges(rng, 40)
    w = _charges(rng, 30)
    lhs = np.vdot(w, direct.direct(s, t, q, kappa))
    rhs = np.vdot(direct.direct_adjoint(s, t, w, kappa), q)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    target = _charges(rng, 30)

    def loss(src):
        return np.sum(np.abs(direct.direct(src, t, q, kappa) - target) ** 2)
    resid = direct.direct(s, t, q, kappa) - target
    g = direct.direct_grad_sources(s, t, q, resid, kappa)
    h = 1e-6
    for j, c in [(0, 0), (5, 1), (17, 2), (39, 0)]:
        sp, sm = s.copy(), s.copy()
        sp[j, c] += h
        sm[j, c] -= h
        fd = (loss(sp) - loss(sm)) / (2 * h)
        assert fd == pytest.approx(g[j, c], rel=1e-6, abs=1e-6)


@pytest.mark.parametrize("kind", ["cube", "two_spheres"])
def test_two_buffer_boxes(kind):
    """Section 3.3.3 with two buffer boxes (|r0| >= 3 a_l): a smaller truncation l per level
    for the same eps, interaction lists over [-5, 5]^3 offsets, neighbour lists over 5^3
    boxes; the apply stays within eps of the direct sum."""
    rng = np.random.default_rng(31)
    if kind == "cube":
        s = t = rng.random((2500, 3))
        kappa, kw = 70.0, dict(depth=3, root=(0, 0, 0, 1.0))
    else:
        s = rng.standard_normal((1500, 3))
        s /= np.linalg.norm(s, axis=1)[:, None]
        t = rng.standard_normal((900, 3))
        t *= 1.5 / np.linalg.norm(t, axis=1)[:, None]
        kappa, kw = 16.0, dict(max_leaf=16)
    q = _charges(rng, len(s))
    p1 = fmm.Plan(s, t, kappa, 1e-6, **kw)
    p2 = fmm.Plan(s, t, kappa, 1e-6, buffer=2, **kw)
    assert p2.lf >= 2
    for l in p2.levels:
        assert p2.levels[l].r0 == 3 * p2.tree.levels[l]['a']
        if l in p1.levels and p1.levels[l].alpha == p2.levels[l].alpha:
            assert p2.levels[l].ell < p1.levels[l].ell
    assert max(len(x) for x in p2.tree.nlist) <= 125
    assert _rel(fmm.apply(p2, q), direct.direct(s, t, q, kappa)) < 1e-6
