"""Double-float arithmetic of the kernels (csrc/df.cuh, green_df in csrc/kernels.cuh), stated
in numpy float32 with single-rounding FMA, against float64 references.  Pins the precision
claims the planner and the near-field policy rely on:

* exp(2 pi i t) by the 1024-entry table, Taylor terms and float32 corrections: absolute error
  below 2^-46 (worst seen about 3 * 2^-48);
* the fused complex product (one two-product sum per component): relative error below 2^-46;
* R and 1/R of the double-float near field (rsqrt seed and one Newton step each): relative
  error below 2^-41 for a seed 2^-22 off (the Newton step leaves about 1.5 x seed error
  squared; worst seen about 2^-42.4).
"""
import numpy as np

f32 = np.float32
N = 1024


def fma(a, b, c):
    # a*b is exact in float64 for float32 inputs; one rounding to float32 of the sum
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def fast_sum(a, b):
    s = f32(a + b)
    return s, f32(b - f32(s - a))


def df(x):
    h = f32(x)
    return h, f32(x - np.float64(h))


def val(a):
    return np.float64(a[0]) + np.float64(a[1])


def df_mul(a, b):
    p = f32(a[0] * b[0])
    e = fma(a[1], b[0], fma(a[0], b[1], fma(a[0], b[0], -p)))
    return fast_sum(p, e)


def df_dot2(a, b, c, d):
    p, q = f32(a[0] * b[0]), f32(c[0] * d[0])
    e = f32(fma(a[0], b[0], -p) + fma(c[0], d[0], -q))
    e = fma(a[0], b[1], fma(a[1], b[0], e))
    e = fma(c[0], d[1], fma(c[1], d[0], e))
    s = two_sum(p, q)
    return fast_sum(s[0], f32(s[1] + e))


def cmul(a, b):
    return (df_dot2(a[0], b[0], (f32(-a[1][0]), f32(-a[1][1])), b[1]), df_dot2(a[0], b[1], a[1], b[0]))


TAB = [(df(np.cos(2 * np.pi * j / N)), df(np.sin(2 * np.pi * j / N))) for j in range(N)]
TWO_PI = (f32(6.2831854820251465), f32(-1.7484555314695172e-07))


def cis_turns(t):
    jf = f32(np.rint(f32(t[0] * f32(N))))
    rr = fast_sum(f32(t[0] - f32(jf * f32(1.0 / N))), t[1])
    x = df_mul(rr, TWO_PI)
    yh = f32(x[0] * x[0])
    ye = fma(f32(x[0] + x[0]), x[1], fma(x[0], x[0], -yh))
    h = f32(f32(-0.5) * yh)
    c = f32(f32(1.0) + h)
    ce = f32(h - f32(c - f32(1.0)))
    cc = fast_sum(c, fma(f32(yh * yh), f32(1.0 / 24.0), fma(f32(-0.5), ye, ce)))
    x3 = f32(x[0] * yh)
    ss = fast_sum(x[0], f32(x[1] + f32(x3 * fma(yh, f32(1.0 / 120.0), f32(-1.0 / 6.0)))))
    return cmul(TAB[int(jf) & (N - 1)], (cc, ss))


def test_cis_absolute_error():
    rng = np.random.default_rng(7)
    worst = 0.0
    for t in rng.uniform(-16, 16, 4000):
        td = df(t)
        tt = val(td)
        re, im = cis_turns(td)
        ref = np.exp(2j * np.pi * (tt - np.rint(tt)))     # reduced first: exact argument
        worst = max(worst, abs(complex(val(re), val(im)) - ref))
    assert worst < 2.0 ** -46, worst


def test_fused_complex_product():
    rng = np.random.default_rng(8)
    worst = 0.0
    for _ in range(4000):
        a = rng.standard_normal(2) * np.exp(rng.uniform(-3, 3))
        b = rng.standard_normal(2) * np.exp(rng.uniform(-3, 3))
        A, B = (df(a[0]), df(a[1])), (df(b[0]), df(b[1]))
        av, bv = complex(val(A[0]), val(A[1])), complex(val(B[0]), val(B[1]))
        re, im = cmul(A, B)
        got = complex(val(re), val(im))
        worst = max(worst, abs(got - av * bv) / (abs(av) * abs(bv)))
    assert worst < 2.0 ** -46, worst


def test_near_field_distance_and_reciprocal():
    rng = np.random.default_rng(9)
    worst_r = worst_inv = 0.0
    for _ in range(4000):
        d = rng.uniform(-1, 1, 3) * np.exp(rng.uniform(-8, 0))
        D = [df(v) for v in d]
        # r2 = d . d as an error-free dot product (df_dot3 of d with itself)
        p = [f32(x[0] * x[0]) for x in D]
        e = f32(f32(fma(D[0][0], D[0][0], -p[0]) + fma(D[1][0], D[1][0], -p[1])) + fma(D[2][0], D[2][0], -p[2]))
        for x in D:
            e = fma(x[0], x[1], fma(x[1], x[0], e))
        a = two_sum(p[0], p[1])
        b = two_sum(a[0], p[2])
        r2 = fast_sum(b[0], f32(f32(a[1] + b[1]) + e))
        y = f32(1.0 / np.sqrt(np.float64(r2[0])) * (1 + 2.0 ** -22))   # a seed off by 2^-22
        r0 = f32(r2[0] * y)
        pp = f32(r0 * r0)
        pe = fma(r0, r0, -pp)
        res = f32(f32(f32(r2[0] - pp) - pe) + r2[1])
        R = fast_sum(r0, f32(res * f32(f32(0.5) * y)))
        q = f32(R[0] * y)
        qe = fma(R[0], y, -q)
        ee = f32(f32(f32(f32(1.0) - q) - qe) - f32(R[1] * y))
        inv = fast_sum(y, f32(y * ee))
        rr = np.sqrt(sum(val(x) ** 2 for x in D))
        worst_r = max(worst_r, abs(val(R) - rr) / rr)
        worst_inv = max(worst_inv, abs(val(inv) - 1 / rr) * rr)
    assert worst_r < 2.0 ** -41 and worst_inv < 2.0 ** -41, (worst_r, worst_inv)


def _turns_f(a, d):
    """The float32-only reduced phase of the float32 levels' S2M / L2T (turns_f), step by step."""
    p = [f32(a[c] * d[c]) for c in range(3)]
    e = [fma(a[c], d[c], -p[c]) for c in range(3)]
    s1, r1 = two_sum(p[0], p[1])
    s2, r2 = two_sum(s1, p[2])
    err = f32(r1 + r2)
    cross = fma(a[0], d[3], fma(a[1], d[4], fma(a[2], d[5], fma(a[3], d[0], fma(a[4], d[1], f32(a[5] * d[2]))))))
    red = f32(s2 - np.rint(s2))
    return f32(red + f32(f32(err + f32(f32(e[0] + e[1]) + e[2])) + cross))


def test_float_phase_of_float32_levels():
    """kappa s.d / (2 pi) reduced to [-1/2, 1/2] from float splits of a = kappa s / (2 pi) and d:
    absolute error below 2^-24 turns (worst seen 2^-26, the rounding of the reduced phase) for phases
    up to 40 turns, the
    range of float32 levels (kappa a_l up to a few hundred at the coarsest level)."""
    rng = np.random.default_rng(7)
    worst = 0.0
    for _ in range(20000):
        s = rng.standard_normal(3)
        s /= np.linalg.norm(s)
        kt = rng.uniform(1.0, 60.0) / (2 * np.pi)
        d = rng.uniform(-1.0, 1.0, 3) * rng.uniform(0.01, 2.0)
        a = kt * s
        af = [f32(x) for x in a] + [f32(a[c] - np.float64(f32(a[c]))) for c in range(3)]
        dfv = [f32(x) for x in d] + [f32(d[c] - np.float64(f32(d[c]))) for c in range(3)]
        exact = float(np.dot(a, d))
        exact -= np.rint(exact)
        got = float(_turns_f(af, dfv))
        diff = abs(got - exact)
        diff = min(diff, abs(diff - 1.0))          # +-1/2 may land on either end
        worst = max(worst, diff)
    assert worst < 2.0 ** -24, worst
