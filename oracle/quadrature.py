"""Truncation, quadrature selection and transfer functions (oracle; test infrastructure only).

Written from Sections 2.1 and 3 of the paper:

* Eq. (EBF)          l ~ kr + C (kr)^(1/3), C = 1.8 d0^(2/3)
* Eq. (CollinoError) closed-form Gegenbauer tail bound (max over the +/- forms)
* Eq. (TransferFn)   T_{l,r0}(s) = (i k / 4 pi) sum_n i^n (2n+1) h_n(k|r0|) P_n(s.r0^)
* Section 3.2        F_n[|sin|] = ((-1)^n + 1) / (pi (1 - n^2))
* Algorithm BMTF     theta band-limited modified transfer function T^{s,L}
* Algorithm Ntheta   N_theta from the bound Eq. (EpsITheta)
* Algorithm Nphi     N_phi(theta_n) from the bound Eq. (EpsIPhi)
* Section 3.3.2      T^{s,LL}: T^{s,L} band-limited per row to N_phi(theta_n)
* Section 3.4        the five-step FFT re-quadrature between two quadratures

Readings where the paper is silent (identical in the product planner, decided
independently there):

* per-level relative target eps_l = eps / 4; absolute threshold eps_l / |r0|
  (|G| ~ 1 / |r0| for the closest far-field pair); d0 = -log10(eps_l);
* |r| = alpha sqrt(3) a_l, |r0| = (b + 1) a_l for b buffer boxes (Section 3.3.3:
  b = 1, the common case, |r0| = 2 a_l; b = 2, |r0| = 3 a_l);
* l: start at the EBF value; if it passes the Collino bound step down while the
  next smaller l still passes, else step up until one passes;
* N_theta^max = N_phi^max = 2l + 64, doubled when nothing below it passes;
* N_phi(theta_n) is the smallest multiple of 4 (>= 4) that passes; rows
  n <= N_theta/4 are searched and mirrored to N_theta/2 - n;
* after each search N_theta is rounded up to 2 * (2^a 3^b 5^c) and N_phi to
  4 * (2^a 3^b 5^c), so that every FFT length factors into 2, 3 and 5;
* re-sampling a length-K sequence to length K' keeps the frequencies
  |k| <= min(ceil(K/2), ceil(K'/2)) - 1 (even lengths drop their Nyquist bin,
  as the truncations of Algorithm BMTF and of T^{s,LL} do).

All arithmetic is float64 / complex128; scipy supplies the special functions.
"""
import math

import numpy as np
from scipy import special as sp

TWO_PI = 2.0 * np.pi
FOUR_PI2 = 4.0 * np.pi * np.pi

# unit round-offs used by the stability rule
U_FP64 = 2.0 ** -53
U_DF = 2.0 ** -48      # float32 pairs (double-float)
U_FP32 = 2.0 ** -24


# --------------------------------------------------------------------------
# special functions (scipy)
# --------------------------------------------------------------------------
def sph_h1(n, x):
    """Spherical Hankel function of the first kind h_n^(1) = j_n + i y_n."""
    return sp.spherical_jn(n, x) + 1j * sp.spherical_yn(n, x)


def i_pow(n):
    """i^n for integer array n, exactly."""
    return np.array([1.0, 1.0j, -1.0, -1.0j])[np.asarray(n) % 4]


# --------------------------------------------------------------------------
# Section 2.1: truncation parameter
# --------------------------------------------------------------------------
def ebf_ell(kr, d0):
    """Eq. (EBF) with C = 1.8 d0^(2/3), rounded up."""
    return int(math.ceil(kr + 1.8 * d0 ** (2.0 / 3.0) * kr ** (1.0 / 3.0)))


def collino_bound(ell, kappa, r, r0):
    """Eq. (CollinoError): closed form of the Gegenbauer tail, max over the +/- forms."""
    vals = []
    for s in (1.0, -1.0):
        br = sph_h1(ell + 1, kappa * r0) * sp.spherical_jn(ell, kappa * r) \
            + s * sph_h1(ell, kappa * r0) * sp.spherical_jn(ell + 1, kappa * r)
        vals.append(kappa * kappa * (r * r0 / (r0 + s * r)) * abs(br))
    return max(vals)


def gegenbauer_tail(ell, kappa, r, r0, sign, nmax):
    """k |sum_{n=l+1}^{nmax} (-sign)^n (2n+1) h_n(k r0) j_n(k r)| (the sum the closed form equals)."""
    n = np.arange(ell + 1, nmax + 1)
    terms = ((-sign) ** n) * (2 * n + 1) * sph_h1(n, kappa * r0) * sp.spherical_jn(n, kappa * r)
    return kappa * abs(np.sum(terms))


def choose_ell(kappa, r, r0, eps_abs, d0):
    """Smallest l near the EBF guess whose Collino bound is <= eps_abs."""
    def passes(l):
        return collino_bound(l, kappa, r, r0) <= eps_abs
    l = max(1, ebf_ell(kappa * r, d0))
    if passes(l):
        while l > 1 and passes(l - 1):
            l -= 1
    else:
        start = l
        while not passes(l):
            l += 1
            if l > start + 2000:
                raise RuntimeError("truncation search did not converge")
    return l


# --------------------------------------------------------------------------
# Eq. (TransferFn) and Section 3.2
# --------------------------------------------------------------------------
def transfer(ell, kappa, r0vec, shat):
    """T_{l,r0}(s) for unit vectors shat[..., 3]."""
    r0vec = np.asarray(r0vec, dtype=np.float64)
    r0 = float(np.sqrt(np.sum(r0vec * r0vec)))
    n = np.arange(ell + 1)
    c = (1j * kappa / (4.0 * np.pi)) * i_pow(n) * (2 * n + 1) * sph_h1(n, kappa * r0)
    t = shat @ (r0vec / r0)
    return np.polynomial.legendre.legval(t, c)


def s_tilde(n):
    """Fourier coefficients of |sin(theta)|: ((-1)^n + 1) / (pi (1 - n^2)); zero for odd n."""
    n = np.asarray(n)
    out = np.zeros(n.shape, dtype=np.float64)
    even = (n % 2) == 0
    ne = n[even].astype(np.float64)
    out[even] = 2.0 / (np.pi * (1.0 - ne * ne))
    return out


def shat_of(theta, phi):
    """Unit vector [cos(phi) sin(theta), sin(phi) sin(theta), cos(theta)]."""
    st = np.sin(theta)
    return np.stack([np.cos(phi) * st, np.sin(phi) * st, np.cos(theta) + 0.0 * phi], axis=-1)


# --------------------------------------------------------------------------
# Algorithm BMTF
# --------------------------------------------------------------------------
def tsl_theta_coeffs(ell, kappa, r0vec, ntheta, phis):
    """Algorithm BMTF, up to the truncation: theta-Fourier coefficients of T^{s,L}.

    Returns (freqs, C) with freqs = -B..B, B = ntheta/2 - 1, and C[freq, p] the
    coefficient of exp(i freq theta) of T^{s,L}(., phis[p]).
    """
    phis = np.atleast_1d(np.asarray(phis, dtype=np.float64))
    m = 2 * ell + 1
    th = TWO_PI * np.arange(m) / m
    shat = shat_of(th[:, None], phis[None, :])            # [m, P, 3]
    half_t = 0.5 * transfer(ell, kappa, r0vec, shat)        # [m, P]
    tc = np.fft.fft(half_t, axis=0) / m                     # exact: degree <= l in theta
    fr = np.arange(-ell, ell + 1)
    tf = tc[fr % m]                                         # [2l+1, P]
    b = ntheta // 2 - 1
    out_fr = np.arange(-b, b + 1)
    conv = s_tilde(out_fr[:, None] - fr[None, :])           # |n - j| <= ntheta/2 + l - 1
    return out_fr, conv @ tf


def tsl_values(ell, kappa, r0vec, ntheta, phis):
    """T^{s,L}(theta_n, phi) on theta_n = 2 pi n / ntheta, n = 0..ntheta-1 (inverse transform)."""
    fr, c = tsl_theta_coeffs(ell, kappa, r0vec, ntheta, phis)
    th = TWO_PI * np.arange(ntheta) / ntheta
    return np.exp(1j * np.outer(th, fr)) @ c


# --------------------------------------------------------------------------
# Algorithms Ntheta and Nphi
# --------------------------------------------------------------------------
def m_index(n_quad, n):
    """M(N, n) of Eq. (EpsITheta)."""
    a = np.abs(n)
    return np.where(a < n_quad / 2.0, n_quad - a, a)


def choose_ntheta(ell, kappa, r, r0, eps_abs):
    """Algorithm Ntheta (before rounding to an FFT-friendly size)."""
    nmax = 2 * ell + 64
    while True:
        fr, c = tsl_theta_coeffs(ell, kappa, (0.0, 0.0, r0), nmax, [0.0])
        tt = np.abs(c[:, 0])
        et = np.abs(sp.jv(np.arange(nmax + 1), kappa * r))
        for nq in range(2 * ell, nmax + 1, 2):
            if np.sum(tt * et[m_index(nq, fr)]) < eps_abs / FOUR_PI2:
                return nq
        nmax *= 2


def choose_nphi(ell, kappa, r, r0, ntheta, eps_abs):
    """Algorithm Nphi (each row before rounding), rows n = 0..ntheta/2."""
    m = 2 * ell + 1
    phis = TWO_PI * np.arange(m) / m
    vals = tsl_values(ell, kappa, (r0, 0.0, 0.0), ntheta, phis)   # [ntheta, m]
    fr = np.arange(-ell, ell + 1)
    half = ntheta // 2
    nphi = np.zeros(half + 1, dtype=np.int64)
    for n in range(half // 2 + 1):
        tt = np.abs((np.fft.fft(vals[n]) / m)[fr % m])
        x = kappa * r * np.sin(TWO_PI * n / ntheta)
        nmax = 2 * ell + 64
        found = 0
        while not found:
            et = np.abs(sp.jv(np.arange(nmax + 1), x))
            for nq in range(4, nmax + 1, 4):
                if np.sum(tt * et[m_index(nq, fr)]) < eps_abs / FOUR_PI2:
                    found = nq
                    break
            nmax *= 2
        nphi[n] = found
    for n in range(half // 2 + 1):
        nphi[half - n] = nphi[n]
    return nphi


def is_235(k):
    for p in (2, 3, 5):
        while k % p == 0:
            k //= p
    return k == 1


def round_fft(n, mult):
    """Smallest mult * (2^a 3^b 5^c) that is >= n."""
    k = max(1, -(-int(n) // mult))
    while not is_235(k):
        k += 1
    return mult * k


# --------------------------------------------------------------------------
# T^{s,LL} (Section 3.3.2)
# --------------------------------------------------------------------------
def tsll(ell, kappa, r0vec, ntheta, nphi):
    """T^{s,LL}_{l,r0} on the half grid (rows n = 0..ntheta/2, N_phi(theta_n) points each), flat."""
    m = 2 * ell + 1
    phis = TWO_PI * np.arange(m) / m
    fr, c = tsl_theta_coeffs(ell, kappa, r0vec, ntheta, phis)   # [2B+1, m]
    mf = np.arange(-ell, ell + 1)
    rows = []
    for n in range(ntheta // 2 + 1):
        th = TWO_PI * n / ntheta
        row_vals = np.exp(1j * th * fr) @ c                 # T^{s,L}(theta_n, 2 pi j / m)
        spec = (np.fft.fft(row_vals) / m)[mf % m]           # |m| <= l, exact
        npn = int(nphi[n])
        b = min(ell, npn // 2 - 1)
        keep = np.abs(mf) <= b
        ph = TWO_PI * np.arange(npn) / npn
        rows.append(np.exp(1j * np.outer(ph, mf[keep])) @ spec[keep])
    return np.concatenate(rows)


# --------------------------------------------------------------------------
# Fourier re-sampling and the five-step re-quadrature (Section 3.4)
# --------------------------------------------------------------------------
def resample(f, kp):
    """Fourier interpolation / anterpolation of the last axis from K to kp samples."""
    f = np.asarray(f, dtype=np.complex128)
    k = f.shape[-1]
    spec = np.fft.fft(f, axis=-1)
    b = min((k + 1) // 2, (kp + 1) // 2) - 1
    fr = np.arange(-b, b + 1)
    g = np.zeros(f.shape[:-1] + (kp,), dtype=np.complex128)
    g[..., fr % kp] = spec[..., fr % k]
    return np.fft.ifft(g, axis=-1) * (kp / k)


class Quadrature:
    """Half-grid uniform quadrature of one level: rows n = 0..ntheta/2, N_phi(theta_n) each."""

    def __init__(self, ell, ntheta, nphi):
        self.ell = int(ell)
        self.ntheta = int(ntheta)
        self.nphi = np.asarray(nphi, dtype=np.int64)
        assert self.nphi.shape[0] == self.ntheta // 2 + 1
        self.offsets = np.concatenate([[0], np.cumsum(self.nphi)]).astype(np.int64)
        self.K = int(self.offsets[-1])
        half = self.ntheta // 2
        th, ph, w = [], [], []
        for n in range(half + 1):
            npn = int(self.nphi[n])
            th.append(np.full(npn, TWO_PI * n / self.ntheta))
            ph.append(TWO_PI * np.arange(npn) / npn)
            mult = 1.0 if n in (0, half) else 2.0
            w.append(np.full(npn, mult * FOUR_PI2 / (self.ntheta * npn)))
        self.theta = np.concatenate(th)
        self.phi = np.concatenate(ph)
        self.w = np.concatenate(w)
        self.shat = shat_of(self.theta, self.phi)

    def rows(self, flat):
        return [flat[..., self.offsets[n]:self.offsets[n + 1]] for n in range(len(self.nphi))]


def requadrature(flat, qa, qb):
    """Section 3.4 steps 1-5: data on quadrature qa (flat half grid) -> quadrature qb.

    flat may carry leading batch axes; the last axis is the half grid of qa.
    """
    flat = np.asarray(flat, dtype=np.complex128)
    lead = flat.shape[:-1]
    big = int(max(qa.nphi.max(), qb.nphi.max()))
    half_a, half_b = qa.ntheta // 2, qb.ntheta // 2
    # step 1: every row of qa to big points
    g = np.zeros(lead + (half_a + 1, big), dtype=np.complex128)
    for n, row in enumerate(qa.rows(flat)):
        g[..., n, :] = resample(row, big)
    # step 2: theta-periodic columns for phi_m, m < big/2
    cols = np.zeros(lead + (big // 2, qa.ntheta), dtype=np.complex128)
    for n in range(qa.ntheta):
        if n <= half_a:
            cols[..., :, n] = g[..., n, :big // 2]
        else:
            cols[..., :, n] = g[..., qa.ntheta - n, big // 2:]
    # step 3: theta re-sampling
    cols = resample(cols, qb.ntheta)
    # step 4: phi-periodic rows of qb
    h = np.zeros(lead + (half_b + 1, big), dtype=np.complex128)
    for n in range(half_b + 1):
        h[..., n, :big // 2] = cols[..., :, n]
        h[..., n, big // 2:] = cols[..., :, (qb.ntheta - n) % qb.ntheta]
    # step 5: every row to N'_phi(theta_n)
    out = [resample(h[..., n, :], int(qb.nphi[n])) for n in range(half_b + 1)]
    return np.concatenate(out, axis=-1)


# --------------------------------------------------------------------------
# one level of the plan
# --------------------------------------------------------------------------
class LevelPlan:
    """l, quadrature and error-model numbers of one level with box size a."""

    def __init__(self, kappa, a, eps_l, alpha, buffer=1):
        self.kappa, self.a, self.eps_l, self.alpha = kappa, a, eps_l, alpha
        self.r = alpha * math.sqrt(3.0) * a
        self.r0 = (buffer + 1.0) * a
        self.eps_abs = eps_l / self.r0
        d0 = -math.log10(eps_l)
        self.ell = choose_ell(kappa, self.r, self.r0, self.eps_abs, d0)
        nt = choose_ntheta(self.ell, kappa, self.r, self.r0, self.eps_abs)
        self.ntheta = round_fft(nt, 2)
        nphi = choose_nphi(self.ell, kappa, self.r, self.r0, self.ntheta, self.eps_abs)
        self.nphi = np.array([round_fft(v, 4) for v in nphi], dtype=np.int64)
        self.quad = Quadrature(self.ell, self.ntheta, self.nphi)
        self.K = self.quad.K

    def rounding_estimate(self, u):
        """Relative round-off of the far-field sum at unit round-off u.

        u * k|r0| * rms_S2(T) * 4 pi / sqrt(K), with the sphere rms of the transfer
        function from the orthogonality of the P_n: 4 pi rms^2 = (k/4pi)^2 4 pi
        sum (2n+1) |h_n(k|r0|)|^2.
        """
        return rounding_estimate(self.ell, self.kappa, self.r0, self.K, u)


def rounding_estimate(ell, kappa, r0, K, u):
    n = np.arange(ell + 1)
    s = np.sum((2 * n + 1) * np.abs(sph_h1(n, kappa * r0)) ** 2)
    return u * kappa * r0 * math.sqrt(s) / math.sqrt(K)


def requadrature_transpose(flat, qa, qb):
    """Transpose of requadrature(., qa, qb): data on quadrature qb -> quadrature qa.

    Each step of Section 3.4 transposed in reverse order.  A one-dimensional re-sampling
    from K to K' points transposes to (K'/K) times the re-sampling from K' to K (the
    band is symmetric in K and K'); step 4's duplication of the pole rows transposes to a
    sum of the two halves, step 2's selection to a scatter with zeros.
    """
    flat = np.asarray(flat, dtype=np.complex128)
    lead = flat.shape[:-1]
    big = int(max(qa.nphi.max(), qb.nphi.max()))
    half_a, half_b = qa.ntheta // 2, qb.ntheta // 2
    # step 5^T: rows of qb, N'_phi(n) -> big, scaled by N'_phi(n) / big
    h = np.zeros(lead + (half_b + 1, big), dtype=np.complex128)
    for n, row in enumerate(qb.rows(flat)):
        h[..., n, :] = resample(row, big) * (row.shape[-1] / big)
    # step 4^T: columns of length ntheta_b, pole rows collect both halves
    cols = np.zeros(lead + (big // 2, qb.ntheta), dtype=np.complex128)
    for t in range(qb.ntheta):
        if t <= half_b:
            cols[..., :, t] += h[..., t, :big // 2]
        if t == 0 or t >= half_b:
            cols[..., :, t] += h[..., (qb.ntheta - t) % qb.ntheta, big // 2:]
    # step 3^T: theta re-sampling ntheta_b -> ntheta_a, scaled by ntheta_b / ntheta_a
    cols = resample(cols, qa.ntheta) * (qb.ntheta / qa.ntheta)
    # step 2^T: back to the half grid of qa, zeros in the second half of the pole rows
    g = np.zeros(lead + (half_a + 1, big), dtype=np.complex128)
    for t in range(half_a + 1):
        g[..., t, :big // 2] = cols[..., :, t]
        if 0 < t < half_a:
            g[..., t, big // 2:] = cols[..., :, qa.ntheta - t]
    # step 1^T: big -> N_phi(theta_n), scaled by big / N_phi(theta_n)
    out = [resample(g[..., n, :], int(qa.nphi[n])) * (big / qa.nphi[n]) for n in range(half_a + 1)]
    return np.concatenate(out, axis=-1)
