"""Minimality pins of Algorithms Ntheta and Nphi (oracle; CPU).

The oracle chooses N_theta and N_phi(theta_n) from the bounds of Eq. EpsITheta and Eq.
EpsIPhi: the smallest admissible size whose bound
    sum_n |T~_n| |J_{M(N, n)}(kappa |r|)| < eps_abs / (4 pi^2)
holds, with M(N, n) = N - |n| for |n| < N/2 and |n| otherwise.  Here the coefficients T~
of the band-limited modified transfer function T^{s,L} (Algorithm BMTF) are computed
independently of the oracle's FFT route: as integrals, by scipy.integrate.quad_vec, of
(1/2)|sin theta| T(s(theta, phi)) against exp(-i f theta) and exp(-i m phi), with T summed
from its Legendre series (Eq. TransferFn) by scipy.special.eval_legendre (the inner phi integral of the N_phi case by
a Gauss-Legendre rule of 4l + 80 nodes, ample for its degree-2l trigonometric integrand; the
outer theta integrals, which carry the kink of |sin|, adaptively).  The pin asserts
that the chosen size passes that bound and the next smaller admissible size (N - 2 for
N_theta, N - 4 for N_phi) fails it, and that a wrong threshold or a wrong M(N, n) planted
in the oracle makes the pin fail.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special as sp

from oracle import quadrature as qd

# (kappa a, eps_l, alpha) at a = 1/2: cases whose N_theta lies above the search start 2l
CASES = [(6.0, 2.5e-7, 0.6), (12.0, 2.5e-5, 0.5), (4.0, 2.5e-9, 0.5)]


def _geometry(ka, eps_l, alpha):
    a = 0.5
    kappa = ka / a
    r = alpha * math.sqrt(3.0) * a
    r0 = 2.0 * a
    eps_abs = eps_l / r0
    ell = qd.choose_ell(kappa, r, r0, eps_abs, -math.log10(eps_l))
    return kappa, r, r0, eps_abs, ell


def _legendre_coeffs(ell, kappa, r0):
    """a_n of T(s) = sum_n a_n P_n(s . r0^): (i kappa / 4 pi) i^n (2n+1) h_n(kappa |r0|)."""
    n = np.arange(ell + 1)
    h = sp.spherical_jn(n, kappa * r0) + 1j * sp.spherical_yn(n, kappa * r0)
    return (1j * kappa / (4.0 * np.pi)) * (1j ** n) * (2 * n + 1) * h


def _t_of(acoef, c):
    """T at cos(angle to r0) = c, summed term by term."""
    n = np.arange(len(acoef))
    return np.sum(acoef * sp.eval_legendre(n, c))


def _cplx_quad(fun, a, b, nout):
    """Integral of a complex vector function over [a, b] (real and imaginary parts stacked)."""
    def g(x):
        v = fun(x)
        return np.concatenate([v.real, v.imag])
    val, _ = integrate.quad_vec(g, a, b, epsabs=0.0, epsrel=1e-13, limit=400)
    return val[:nout] + 1j * val[nout:]


def _over_theta(fun, nout):
    """(1/2 pi) times the integral over [0, 2 pi], split at the kink of |sin| at pi."""
    return (_cplx_quad(fun, 0.0, np.pi, nout) + _cplx_quad(fun, np.pi, 2 * np.pi, nout)) / (2 * np.pi)


def _m_index(nq, n):
    a = np.abs(n)
    return np.where(2 * a < nq, nq - a, a)


def _bound(tt, freqs, nq, x):
    return float(np.sum(tt * np.abs(sp.jv(_m_index(nq, freqs), x))))


def theta_coefficients(ell, kappa, r0, band):
    """|T~_f|, f = -band..band, of T^{s,L}(theta, 0) for r0 along z, by quadrature."""
    acoef = _legendre_coeffs(ell, kappa, r0)
    f = np.arange(-band, band + 1)

    def integrand(th):
        return 0.5 * abs(math.sin(th)) * _t_of(acoef, math.cos(th)) * np.exp(-1j * f * th)
    return f, np.abs(_over_theta(integrand, len(f)))


def phi_coefficients(ell, kappa, r0, ntheta, rows):
    """|T~_m(theta_n)|, |m| <= l, of T^{s,L}(theta_n, phi) for r0 along x, by quadrature:
    C[f, m] = (1/2pi)^2 double integral of (1/2)|sin t| T(s(t, p)) exp(-i f t - i m p),
    |f| <= ntheta/2 - 1 (the theta band of T^{s,L}), then sum_f C[f, m] exp(i f theta_n)."""
    acoef = _legendre_coeffs(ell, kappa, r0)
    m = np.arange(-ell, ell + 1)
    band = ntheta // 2 - 1
    f = np.arange(-band, band + 1)

    xg, wg = np.polynomial.legendre.leggauss(4 * ell + 80)
    ph = np.pi * (xg + 1.0)                   # nodes on [0, 2 pi], weights pi * wg
    wph = np.pi * wg
    n = np.arange(ell + 1)
    emph = np.exp(-1j * np.outer(m, ph))      # [m, nodes]

    def phi_coeffs(th):
        tvals = acoef @ sp.eval_legendre(n[:, None], math.sin(th) * np.cos(ph)[None, :])
        return emph @ (wph * tvals) / (2 * np.pi)

    def outer(th):
        return np.outer(0.5 * abs(math.sin(th)) * np.exp(-1j * f * th), phi_coeffs(th)).ravel()
    C = _over_theta(outer, len(f) * len(m)).reshape(len(f), len(m))
    out = {}
    for n in rows:
        th_n = 2 * np.pi * n / ntheta
        out[n] = np.abs(np.exp(1j * f * th_n) @ C)
    return m, out


def ntheta_pin(case):
    """(chosen, passes, next smaller fails) for the oracle's raw N_theta."""
    kappa, r, r0, eps_abs, ell = _geometry(*case)
    nq = qd.choose_ntheta(ell, kappa, r, r0, eps_abs)
    band = (2 * ell + 64) // 2 - 1            # N^max = 2l + 64 (the oracle's first search band)
    assert nq <= 2 * ell + 64
    f, tt = theta_coefficients(ell, kappa, r0, band)
    thr = eps_abs / (4.0 * np.pi ** 2)
    ok = _bound(tt, f, nq, kappa * r) < thr
    smaller_fails = nq - 2 < 2 * ell or _bound(tt, f, nq - 2, kappa * r) >= thr
    return nq, ok, smaller_fails


def nphi_pin(case, tt_cache={}):
    """Per searched row: (row, chosen N_phi, passes, N_phi - 4 fails)."""
    kappa, r, r0, eps_abs, ell = _geometry(*case)
    ntheta = qd.round_fft(qd.choose_ntheta(ell, kappa, r, r0, eps_abs), 2)
    nphi = qd.choose_nphi(ell, kappa, r, r0, ntheta, eps_abs)
    rows = list(range(ntheta // 4 + 1))
    key = case
    if key not in tt_cache:
        tt_cache[key] = phi_coefficients(ell, kappa, r0, ntheta, rows)
    m, tt = tt_cache[key]
    thr = eps_abs / (4.0 * np.pi ** 2)
    out = []
    for n in rows:
        x = kappa * r * math.sin(2 * np.pi * n / ntheta)
        npn = int(nphi[n])
        ok = _bound(tt[n], m, npn, x) < thr
        smaller_fails = npn - 4 < 4 or _bound(tt[n], m, npn - 4, x) >= thr
        out.append((n, npn, ok, smaller_fails))
    return out


@pytest.mark.parametrize("case", CASES)
def test_ntheta_is_the_smallest_passing_size(case):
    nq, ok, smaller_fails = ntheta_pin(case)
    kappa, r, r0, eps_abs, ell = _geometry(*case)
    assert nq > 2 * ell          # the case exercises the search beyond its start
    assert ok, (case, nq)
    assert smaller_fails, (case, nq)


@pytest.mark.parametrize("case", CASES)
def test_nphi_is_the_smallest_passing_size(case):
    rows = nphi_pin(case)
    assert any(npn > 4 for _, npn, _, _ in rows)
    for n, npn, ok, smaller_fails in rows:
        assert ok, (case, n, npn)
        assert smaller_fails, (case, n, npn)


def test_pins_catch_a_wrong_threshold(monkeypatch):
    """A 2 pi threshold (the prefactor printed in Eq. EpsIPhi) in place of 4 pi^2 lets
    smaller sizes through; the independent bound must reject them."""
    monkeypatch.setattr(qd, "FOUR_PI2", 2.0 * np.pi)
    _, ok, _ = ntheta_pin(CASES[0])
    assert not ok
    rows = nphi_pin(CASES[0], tt_cache={})
    assert not all(ok for _, _, ok, _ in rows)


def test_pins_catch_a_wrong_m_index(monkeypatch):
    """M(N, n) = N - |n| for every n (dropping the |n| >= N/2 branch) changes the chosen
    sizes; the independent bound must notice."""
    monkeypatch.setattr(qd, "m_index", lambda nq, n: nq - np.abs(n))
    res = [ntheta_pin(c) for c in CASES]
    assert not all(ok and fails for _, ok, fails in res)
