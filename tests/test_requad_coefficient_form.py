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


def coefficient_requad_transpose(yflat, qa, qb):
    """Transpose of coefficient_requad(., qa, qb) as the transposed kernels compute it
    (k_requad_spec_ct, k_requad_spec_cols_t, k_requad_spec_at_*): grid b -> grid a."""
    big = int(max(qa.nphi.max(), qb.nphi.max()))
    nta, ntb = qa.ntheta, qb.ntheta
    ha, hbr = nta // 2, ntb // 2
    GB = np.zeros((hbr + 1, big), complex)                  # C'^T: unnormalised inverse FFT
    for n, row in enumerate(qb.rows(yflat)):
        ln = len(row)
        b = _band(big, ln)
        z = np.fft.ifft(row) * ln
        for j in range(ln):
            f = _freq(j, ln)
            if -b <= f <= b:
                GB[n, (f + big) % big] = z[j]
    GA = np.zeros((ha + 1, big), complex)                   # B'^T
    for c in range(big // 2):
        se, so = (c, big - 1 - c) if c % 2 == 0 else (big - 1 - c, c)
        y = np.zeros(ntb, complex)
        for m in range(ntb):
            if m in (0, hbr):
                y[m] = GB[m, se]
            elif m < hbr:
                y[m] = 0.5 * (GB[m, se] + GB[m, so])
            else:
                y[m] = 0.5 * (GB[ntb - m, se] - GB[ntb - m, so])
        h = _resample(y, nta) * (ntb / nta)
        for u in range(ha + 1):
            hm = h[nta - u] if 0 < u < ha else 0.0
            GA[u, se], GA[u, so] = h[u] + hm, h[u] - hm
    out = []                                                # A'^T: forward FFT / N_phi
    for t in range(ha + 1):
        ln = int(qa.nphi[t])
        b = _band(ln, big)
        buf = np.zeros(ln, complex)
        for j in range(ln):
            f = _freq(j, ln)
            if -b <= f <= b:
                buf[j] = GA[t, (f + big) % big]
        out.append(np.fft.fft(buf) / ln)
    return np.concatenate(out)


@pytest.mark.parametrize("kappa,sizes", [(40.0, (2.0 / 8, 2.0 / 4)), (30.0, (2.0 / 16, 2.0 / 8))])
def test_transposed_passes_are_the_transpose(kappa, sizes):
    qa, qb = (oq.LevelPlan(kappa, a, 1e-4, 0.8).quad for a in sizes)
    assert qa.ntheta != qb.ntheta
    F = np.array([coefficient_requad(e, qa, qb) for e in np.eye(qa.K)]).T    # K_b x K_a
    rng = np.random.default_rng(11)
    y = rng.standard_normal(qb.K) + 1j * rng.standard_normal(qb.K)
    want = F.T @ y
    got = coefficient_requad_transpose(y, qa, qb)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))
