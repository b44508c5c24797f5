"""Pins of the oracle's Fourier building blocks (Section 3.1 of the paper).

Independent checks: printed numbers of Figure SINFspec, closed forms
(Fourier series of |sin|, the toy integral sin(64)/16, Jacobi-Anger), numerical
integration with scipy.integrate.quad, and exactness of Fourier re-sampling on
band-limited trigonometric polynomials.
"""
import os

import numpy as np
import pytest
from scipy import integrate
from scipy.special import jv

from oracle import quadrature as qd

GOLDEN = os.path.join(os.path.dirname(__file__), 'golden')


def test_sinfspec_printed_values():
    """Figure SINFspec: spectrum of cos(64 cos theta) from 256 samples (printed values)."""
    data = np.loadtxt(os.path.join(GOLDEN, 'sinfspec.txt'))
    th = qd.TWO_PI * np.arange(256) / 256
    spec = np.fft.fft(np.cos(64.0 * np.cos(th))) / 256
    for n, val in data:
        got = abs(spec[int(n) % 256])
        assert got == pytest.approx(val, rel=6e-5, abs=1e-15), n
    # and the printed values are |J_n(64)| (Jacobi-Anger, Eq. PlaneWaveSpec)
    for n, val in data:
        assert abs(jv(int(n), 64.0)) == pytest.approx(val, rel=6e-5, abs=1e-15)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 7, 10, 31, 64])
def test_abs_sin_series(n):
    """Section 3.2: F_n[|sin|] = ((-1)^n + 1) / (pi (1 - n^2)), against quad on the two smooth halves."""
    def part(f):
        a = integrate.quad(lambda t: f(t) * np.sin(t), 0, np.pi, limit=200, epsabs=1e-14)[0]
        b = integrate.quad(lambda t: f(t) * (-np.sin(t)), np.pi, 2 * np.pi, limit=200, epsabs=1e-14)[0]
        return (a + b) / (2 * np.pi)
    re = part(lambda t: np.cos(n * t))
    im = -part(lambda t: np.sin(n * t))
    assert qd.s_tilde(np.array([n]))[0] == pytest.approx(re, abs=1e-12)
    assert abs(im) < 1e-12
    assert qd.s_tilde(np.array([-n]))[0] == qd.s_tilde(np.array([n]))[0]


def _filtered_toy(nb):
    """Section 3.1.2 toy: |sin| band-limited to |n| <= nb, K = 2 nb + 1 points."""
    k = 2 * nb + 1
    th = qd.TWO_PI * np.arange(k) / k
    fr = np.arange(-nb, nb + 1)
    f_n = np.real(np.exp(1j * np.outer(th, fr)) @ qd.s_tilde(fr))
    return qd.TWO_PI / k * np.sum(f_n * np.cos(64.0 * np.cos(th)))


def test_toy_integral_closed_form():
    exact = np.sin(64.0) / 16.0
    quad_val = integrate.quad(lambda t: abs(np.sin(t)) * np.cos(64 * np.cos(t)), 0, 2 * np.pi,
                              points=[np.pi], limit=500, epsabs=1e-14)[0]
    assert quad_val == pytest.approx(exact, abs=1e-12)
    # Figure SINConv: the filtered quadrature converges super-exponentially past N ~ 66
    errs = {nb: abs(_filtered_toy(nb) - exact) / abs(exact) for nb in (40, 60, 80, 108, 200)}
    assert errs[40] > 1e-3
    assert errs[80] < 1e-6
    assert errs[108] < 1e-13
    assert errs[200] < 1e-13


def test_trapezoid_is_slow():
    """Figure SINConv: plain trapezoid converges like 1/K^2 (|sin| is only C^0)."""
    exact = np.sin(64.0) / 16.0
    def trap(k):
        th = qd.TWO_PI * np.arange(k) / k
        return qd.TWO_PI / k * np.sum(np.abs(np.sin(th)) * np.cos(64 * np.cos(th)))
    e1 = abs(trap(1001) - exact)
    e2 = abs(trap(2001) - exact)
    assert 1e-7 < e1 < 1e-3
    assert 2.5 < e1 / e2 < 6.0


def test_jacobi_anger():
    """Eq. PlaneWaveSpec: Fourier coefficients of exp(i x cos(theta)) are i^n J_n(x)."""
    x = 23.7
    k = 128
    th = qd.TWO_PI * np.arange(k) / k
    spec = np.fft.fft(np.exp(1j * x * np.cos(th))) / k
    n = np.arange(-50, 51)
    assert np.max(np.abs(spec[n % k] - qd.i_pow(n) * jv(n, x))) < 1e-13


def _trig(coef, fr, k):
    th = qd.TWO_PI * np.arange(k) / k
    return np.exp(1j * np.outer(th, fr)) @ coef


@pytest.mark.parametrize("k,kp", [(24, 40), (40, 24), (25, 36), (36, 36), (60, 120)])
def test_resample_exact_on_band(k, kp):
    rng = np.random.default_rng(5)
    b = min((k + 1) // 2, (kp + 1) // 2) - 1
    fr = np.arange(-b, b + 1)
    coef = rng.standard_normal(len(fr)) + 1j * rng.standard_normal(len(fr))
    f = _trig(coef, fr, k)
    g = qd.resample(f, kp)
    assert np.max(np.abs(g - _trig(coef, fr, kp))) < 1e-12


def test_anterpolation_truncates_and_is_adjoint():
    rng = np.random.default_rng(6)
    k, kp = 48, 20
    f = rng.standard_normal(k) + 1j * rng.standard_normal(k)
    g = qd.resample(f, kp)
    spec = np.fft.fft(f) / k
    fr = np.arange(-(kp // 2 - 1), kp // 2)
    assert np.max(np.abs(g - _trig(spec[fr % k], fr, kp))) < 1e-12
    # anterp_{K->K'} = (K'/K) interp_{K'->K}^T under the 1/K quadrature weights
    A = np.stack([qd.resample(e, kp) for e in np.eye(k)], axis=1)      # K' x K
    B = np.stack([qd.resample(e, k) for e in np.eye(kp)], axis=1)      # K x K'
    assert np.max(np.abs(A - (kp / k) * B.T)) < 1e-13
