"""Pins of the oracle's truncation, transfer function and quadrature (Sections 2.1, 3.3, 3.4).

Independent checks: closed forms (h_0, the Gegenbauer series summing to the
kernel, the Funk-Hecke identity by Gauss-Legendre quadrature), numerical
Fourier coefficients by scipy.integrate.quad, the tail sum the Collino closed
form equals, the paper's own error claims (eps_T within ~2x of the target,
quadrature ratio near 2/pi), and exact band-limited re-quadrature.
"""
import numpy as np
import pytest
from scipy import integrate
from scipy.special import spherical_jn

from oracle import quadrature as qd


def test_hankel_closed_form():
    x = np.array([0.3, 1.0, 7.5, 40.0])
    assert np.allclose(qd.sph_h1(0, x), -1j * np.exp(1j * x) / x, rtol=1e-14)
    assert np.allclose(qd.sph_h1(1, x), -np.exp(1j * x) * (x + 1j) / x ** 2, rtol=1e-14)


@pytest.mark.parametrize("ell,kappa,a", [(30, 10.0, 1.0), (45, 20.0, 0.7), (12, 3.0, 1.0)])
def test_collino_closed_form_equals_tail_sum(ell, kappa, a):
    r, r0 = 0.8 * np.sqrt(3) * a, 2 * a
    for s in (1.0, -1.0):
        tail = qd.gegenbauer_tail(ell, kappa, r, r0, s, ell + 70)
        br = qd.sph_h1(ell + 1, kappa * r0) * spherical_jn(ell, kappa * r) \
            + s * qd.sph_h1(ell, kappa * r0) * spherical_jn(ell + 1, kappa * r)
        closed = kappa ** 2 * (r * r0 / (r0 + s * r)) * abs(br)
        assert closed == pytest.approx(tail, rel=1e-9)
    assert qd.collino_bound(ell, kappa, r, r0) == pytest.approx(
        max(qd.gegenbauer_tail(ell, kappa, r, r0, 1.0, ell + 70),
            qd.gegenbauer_tail(ell, kappa, r, r0, -1.0, ell + 70)), rel=1e-9)


def _sphere_quad(nlat):
    """Gauss-Legendre in cos(theta) x uniform phi: exact for degree < nlat spherical polynomials."""
    z, wz = np.polynomial.legendre.leggauss(nlat)
    phi = qd.TWO_PI * np.arange(2 * nlat) / (2 * nlat)
    zz, pp = np.meshgrid(z, phi, indexing='ij')
    st = np.sqrt(1 - zz ** 2)
    shat = np.stack([np.cos(pp) * st, np.sin(pp) * st, zz], axis=-1).reshape(-1, 3)
    w = (wz[:, None] * np.full(phi.shape, qd.TWO_PI / (2 * nlat))[None, :]).reshape(-1)
    return shat, w


def test_transfer_funk_hecke_and_gegenbauer():
    """int_S2 exp(i k s.r) T_{l,r0}(s) dS = truncated Eq. Gegenbauer, which tends to the kernel."""
    kappa, ell = 20.0, 30          # l < k|r0|: outside the low-frequency breakdown
    r0v = np.array([1.2, -0.9, 1.5])
    rv = np.array([0.31, 0.22, -0.4])
    shat, w = _sphere_quad(120)
    lhs = np.sum(w * np.exp(1j * kappa * (shat @ rv)) * qd.transfer(ell, kappa, r0v, shat))
    r, r0 = np.linalg.norm(rv), np.linalg.norm(r0v)
    n = np.arange(ell + 1)
    t = rv @ r0v / (r * r0)
    geg = 1j * kappa * np.sum((-1.0) ** n * (2 * n + 1) * qd.sph_h1(n, kappa * r0)
                              * spherical_jn(n, kappa * r) * np.polynomial.legendre.legval(t, np.eye(ell + 1)))
    assert abs(lhs - geg) < 1e-11 * abs(geg)
    d = np.linalg.norm(rv + r0v)
    assert abs(geg - np.exp(1j * kappa * d) / d) < 1e-10


@pytest.mark.parametrize("n", [0, 1, 2, 5, 13, 30])
def test_bmtf_coefficients_against_quad(n):
    """Algorithm BMTF gives the exact low theta-frequencies of 1/2 T |sin(theta)|."""
    ell, kappa = 12, 5.0
    r0v = np.array([0.0, 1.0, 2.0])
    phi = 0.7
    fr, c = qd.tsl_theta_coeffs(ell, kappa, r0v, 64, [phi])
    def f(t):
        return 0.5 * qd.transfer(ell, kappa, r0v, qd.shat_of(np.array([t]), np.array([phi])))[0] * abs(np.sin(t))
    def coef(part):
        g = (lambda t: part(f(t) * np.exp(-1j * n * t)))
        return (integrate.quad(g, 0, np.pi, limit=400, epsabs=1e-13)[0]
                + integrate.quad(g, np.pi, 2 * np.pi, limit=400, epsabs=1e-13)[0]) / qd.TWO_PI
    want = coef(np.real) + 1j * coef(np.imag)
    got = c[list(fr).index(n), 0]
    assert abs(got - want) < 1e-10 * max(1.0, abs(want))


def test_tsl_sphere_symmetry():
    """Eq. NumSphereSym: f(theta_n, phi_m) = f(theta_{N-n}, phi_{m+N/2}) for T^{s,L}."""
    ell, kappa, nt, nphi = 10, 4.0, 30, 24
    phis = qd.TWO_PI * np.arange(nphi) / nphi
    v = qd.tsl_values(ell, kappa, (2.0, 1.0, -1.0), nt, phis)
    for n in range(nt):
        for m in range(nphi):
            assert abs(v[n, m] - v[(nt - n) % nt, (m + nphi // 2) % nphi]) < 1e-12 * np.max(np.abs(v))


def _full_grid_sum(lp, rv, r0v):
    """Eq. eps_T quadrature sum over the half grid with folded weights."""
    q = lp.quad
    t = qd.tsll(lp.ell, lp.kappa, r0v, lp.ntheta, lp.nphi)
    return np.sum(q.w * np.exp(1j * lp.kappa * (q.shat @ rv)) * t)


@pytest.mark.parametrize("kappa,buffer", [(20.0, 1), (40.0, 1), (20.0, 2), (40.0, 2)])   # outside the breakdown
def test_total_error_within_target(kappa, buffer):
    """Section 3.5.1: eps_T of the worst-case directions stays within ~2x of the target, with
    one buffer box (|r0| = 2a) and with two (|r0| = 3a, Section 3.3.3)."""
    a = 1.0
    eps_l = 1e-6
    lp = qd.LevelPlan(kappa, a, eps_l, 0.8, buffer)
    r = lp.r
    worst = 0.0
    for r0dir, rdirs in (((0, 0, 1), [(0, 0, 1), (0, 0, -1), (1, 0, 0)]),
                         ((1, 0, 0), [(1, 0, 0), (-1, 0, 0), (0, 1, 1)])):
        r0v = (buffer + 1) * a * np.array(r0dir, dtype=float)
        for rd in rdirs:
            rv = r * np.array(rd, dtype=float) / np.linalg.norm(rd)
            d = np.linalg.norm(rv + r0v)
            err = abs(np.exp(1j * kappa * d) / d - _full_grid_sum(lp, rv, r0v))
            worst = max(worst, err)
    assert worst < 2.0 * lp.eps_abs


def test_total_error_tends_to_gegenbauer():
    """Section 3.5.2 (Figure GegError_Quad): enlarging the quadrature leaves only eps_G."""
    kappa, a = 10.0, 1.0
    r0v = np.array([0.0, 0.0, 2.0])
    rv = np.array([0.0, 0.0, 0.8 * np.sqrt(3)])
    ell = 22
    n = np.arange(ell + 1)
    rr, r0 = np.linalg.norm(rv), 2.0
    geg = 1j * kappa * np.sum((-1.0) ** n * (2 * n + 1) * qd.sph_h1(n, kappa * r0) * spherical_jn(n, kappa * rr))
    errs = []
    for nt, nph in ((40, 40), (50, 52), (60, 60), (80, 80), (120, 120)):
        quad = qd.Quadrature(ell, nt, np.full(nt // 2 + 1, nph))
        t = qd.tsll(ell, kappa, r0v, nt, quad.nphi)
        s = np.sum(quad.w * np.exp(1j * kappa * (quad.shat @ rv)) * t)
        errs.append(abs(s - geg) / abs(geg))
    assert errs[0] > 1e-3 and errs[1] < errs[0] * 1e-2 and errs[2] < errs[1] * 1e-2
    assert errs[3] < 1e-12 and errs[4] < 1e-12


def test_quadrature_size_ratio():
    """Section 3.3.4 / Figure QuadSize: K / 2(l+1)^2 lies well below 1 and drifts towards 2/pi."""
    ratios = []
    for kappa in (8.0, 32.0, 64.0):
        lp = qd.LevelPlan(kappa, 1.0, 1e-4, 0.8)
        ratios.append(lp.K / (2.0 * (lp.ell + 1) ** 2))
    assert all(0.55 < x < 1.0 for x in ratios)
    assert ratios[-1] < 0.8


def _sym_function(nt_band, np_band, rng):
    """Random trig polynomial with Eq. FourierSphereSym: c_{n,m} = (-1)^m c_{-n,m}."""
    c = {}
    for m in range(-np_band, np_band + 1):
        for n in range(0, nt_band + 1):
            v = rng.standard_normal() + 1j * rng.standard_normal()
            c[(n, m)] = v
            c[(-n, m)] = v * (-1) ** m if n else (v if m % 2 == 0 else 0.0)
    def f(theta, phi):
        out = np.zeros(np.broadcast(theta, phi).shape, dtype=complex)
        for (n, m), v in c.items():
            out += v * np.exp(1j * (n * theta + m * phi))
        return out
    return f


def test_requadrature_exact_on_band_limited_data():
    """Section 3.4: the five-step re-quadrature is exact for band-limited spherical data."""
    rng = np.random.default_rng(3)
    f = _sym_function(6, 7, rng)
    qa = qd.Quadrature(8, 18, np.array([4, 16, 20, 20, 24, 20, 20, 16, 16, 4])[:10])
    qb = qd.Quadrature(10, 24, np.array([4, 16, 20, 24, 24, 28, 28, 24, 24, 20, 20, 16, 4])[:13])
    # make qa resolve the band: rows need N_phi >= 2*7+2 except the poles (f is pi-periodic there)
    qa = qd.Quadrature(8, 18, np.array([16] + [16] * 8 + [16]))
    da = f(qa.theta, qa.phi)
    db = qd.requadrature(da, qa, qd.Quadrature(10, 24, np.full(13, 20)))
    qb = qd.Quadrature(10, 24, np.full(13, 20))
    assert np.max(np.abs(db - f(qb.theta, qb.phi))) < 1e-12 * np.max(np.abs(da))
    back = qd.requadrature(db, qb, qa)
    assert np.max(np.abs(back - da)) < 1e-12 * np.max(np.abs(da))
    # quadrature sums agree
    assert abs(np.sum(qa.w * da) - np.sum(qb.w * db)) < 1e-12 * np.sum(np.abs(qa.w * da))


def test_requadrature_transpose_is_the_matrix_transpose():
    """Section 3.4 re-quadrature: the transposed pipeline equals the explicit matrix transpose."""
    qa = qd.Quadrature(6, 12, np.array([4, 8, 12, 12, 12, 8, 4]))
    qb = qd.Quadrature(8, 16, np.array([4, 8, 12, 16, 16, 16, 12, 8, 4]))
    for x, y in ((qa, qb), (qb, qa)):
        A = np.stack([qd.requadrature(e, x, y) for e in np.eye(x.K)], axis=1)          # K_y x K_x
        At = np.stack([qd.requadrature_transpose(e, x, y) for e in np.eye(y.K)], axis=1)  # K_x x K_y
        assert np.max(np.abs(At - A.T)) < 1e-13
