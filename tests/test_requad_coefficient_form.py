"""The forward re-quadrature kernels run Section 3.4's theta steps on phi-Fourier
coefficients (k_requad_spec_*).  This CPU test states that pipeline in numpy and checks
it against the oracle's five-step re-quadrature (sample form):

* on signatures - plane-wave sums, whose pole rows are constant in phi - the two are the
  same map to float64 round-off, for up- and down-going level pairs;
* on arbitrary data whose pole rows vary in phi they differ: the claim is limited to
  signatures, which is what every S2M, M2L and shift output is.
"""
import numpy as np
import pytest

from oracle import quadrature as oq


def _band(n, npr):
    return min((n + 1) // 2, (npr + 1) // 2) - 1


def _freq(j, n):
    return j if 2 * j <= n else j - n


def _resample(x, npr):
    n = len(x)
    X = np.fft.fft(x) / n
    b = _band(n, npr)
    o = np.zeros(npr, complex)
    for j in range(npr):
        f = _freq(j, npr)
        if -b <= f <= b:
            o[j] = X[(f + n) % n]
    return np.fft.ifft(o) * npr


def coefficient_requad(flat, qa, qb):
    big = int(max(qa.nphi.max(), qb.nphi.max()))
    nta, ntb = qa.ntheta, qb.ntheta
    ha, hbr = nta // 2, ntb // 2
    # A': each row's band-limited coefficients in slot (f + big) % big
    GA = np.zeros((ha + 1, big), complex)
    for t, row in enumerate(qa.rows(flat)):
        n = len(row)
        X = np.fft.fft(row) / n
        b = _band(n, big)
        for j in range(big):
            f = _freq(j, big)
            if -b <= f <= b:
                GA[t, j] = X[(f + n) % n]
    # B': slots c and big-1-c (opposite parity) share one theta circle
    GB = np.zeros((hbr + 1, big), complex)
    for c in range(big // 2):
        se, so = (c, big - 1 - c) if c % 2 == 0 else (big - 1 - c, c)
        h = np.array([GA[t, se] + GA[t, so] if t <= ha else GA[nta - t, se] - GA[nta - t, so]
                      for t in range(nta)])
        y = _resample(h, ntb)
        for n in range(hbr + 1):
            ym = y[(ntb - n) % ntb]
            GB[n, se], GB[n, so] = 0.5 * (y[n] + ym), 0.5 * (y[n] - ym)
    # C': each output row from its band of coefficients
    out = []
    for n in range(hbr + 1):
        ln = int(qb.nphi[n])
        b = _band(big, ln)
        buf = np.zeros(ln, complex)
        for j in range(ln):
            f = _freq(j, ln)
            if -b <= f <= b:
                buf[j] = GB[n, (f + big) % big]
        out.append(np.fft.ifft(buf) * ln)
    return np.concatenate(out)


LEVELS = {27: 2.0 / 16, 52: 2.0 / 8, 70: 2.0 / 4}   # box sizes of the 262k-sphere levels (kappa 64)


@pytest.mark.parametrize("pair", [(27, 52), (52, 70), (52, 27), (70, 52)])
def test_same_map_on_signatures(pair):
    la, lb = (oq.LevelPlan(64.0, LEVELS[v], 2.5e-7, 0.8) for v in pair)
    qa, qb = la.quad, lb.quad
    rng = np.random.default_rng(sum(pair))
    d = rng.uniform(-0.5, 0.5, (40, 3)) * la.a
    q = rng.standard_normal(40) + 1j * rng.standard_normal(40)
    x = np.exp(1j * 64.0 * qa.shat @ d.T) @ q                  # a signature on grid a
    a = oq.requadrature(x, qa, qb)
    b = coefficient_requad(x, qa, qb)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))


def test_differs_when_pole_rows_vary():
    la, lb = (oq.LevelPlan(64.0, LEVELS[v], 2.5e-7, 0.8) for v in (27, 52))
    qa, qb = la.quad, lb.quad
    rng = np.random.default_rng(3)
    x = rng.standard_normal(qa.K) + 1j * rng.standard_normal(qa.K)
    a = oq.requadrature(x, qa, qb)
    b = coefficient_requad(x, qa, qb)
    assert np.max(np.abs(a - b)) > 1e-3 * np.max(np.abs(a))
    # making the pole rows constant restores agreement on the rest of the pipeline
    rows = qa.rows(x)
    x2 = x.copy()
    for n in (0, qa.ntheta // 2):
        x2[qa.offsets[n]:qa.offsets[n + 1]] = rows[n][0]
    # not a signature elsewhere, but the only difference left is in how the pole rows are read
    a2, b2 = oq.requadrature(x2, qa, qb), coefficient_requad(x2, qa, qb)
    assert np.max(np.abs(a2 - b2)) <= 1e-12 * np.max(np.abs(a2))
