// Double-float ("df") arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2, both float32,
// about 48 significant bits.  Built from error-free transformations: Knuth's TwoSum,
// Dekker's Fast2Sum and the FMA form of Dekker's exact product.  Every step uses the
// _rn intrinsics so the compiler cannot contract or reassociate it.
//
// cis_turns_big(t) = exp(2 pi i t): reduction by a 1024-entry table of exp(2 pi i j / 1024)
// (stored as df pairs), Taylor polynomials of sin and cos on |x| <= pi/1024, then one complex
// df product.
#pragma once
#include <cuda_runtime.h>

#include "cx.cuh"

namespace hfmm {

struct df {
    float hi, lo;
    df() = default;
    __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ explicit df(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
    __host__ __device__ explicit operator float() const { return hi + lo; }
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ df df_fast_sum(float a, float b) {  // |a| >= |b|
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}
__device__ __forceinline__ df df_add(df a, df b) {
    df s = df_two_sum(a.hi, b.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return df_fast_sum(s.hi, e);
}
// a + b when |a| >= |b| (Dekker's Fast2Sum on the leading parts)
__device__ __forceinline__ df df_add_big(df a, df b) {
    float s = __fadd_rn(a.hi, b.hi);
    float e = __fadd_rn(__fsub_rn(b.hi, __fsub_rn(s, a.hi)), __fadd_rn(a.lo, b.lo));
    return df_fast_sum(s, e);
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_mul(df a, df b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_sum(p, e);
}
__device__ __forceinline__ df df_mul_f(df a, float b) {
    float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return df_fast_sum(p, e);
}
__host__ __device__ __forceinline__ df df_from_double(double x) {
    float h = (float)x;
    return {h, (float)(x - (double)h)};
}
__host__ __device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

struct cdf {
    df x, y;
};

// arithmetic operators so that complex and FFT templates instantiate for df
__device__ __forceinline__ df operator+(df a, df b) { return df_add(a, b); }
__device__ __forceinline__ df operator-(df a, df b) { return df_sub(a, b); }
__device__ __forceinline__ df operator-(df a) { return df_neg(a); }
__device__ __forceinline__ df operator*(df a, df b) { return df_mul(a, b); }
__device__ __forceinline__ df& operator+=(df& a, df b) { a = df_add(a, b); return a; }
__device__ __forceinline__ df& operator-=(df& a, df b) { a = df_sub(a, b); return a; }
// a b + c d: both Dekker products and their exact FMA errors, one Knuth sum of the leading
// parts, every small term gathered in float32, one renormalisation
__device__ __forceinline__ df df_dot2(df a, df b, df c, df d) {
    const float p = __fmul_rn(a.hi, b.hi), q = __fmul_rn(c.hi, d.hi);
    float e = __fadd_rn(__fmaf_rn(a.hi, b.hi, -p), __fmaf_rn(c.hi, d.hi, -q));
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    e = __fmaf_rn(c.hi, d.lo, __fmaf_rn(c.lo, d.hi, e));
    const df s = df_two_sum(p, q);
    return df_fast_sum(s.hi, __fadd_rn(s.lo, e));
}
__device__ __forceinline__ cdf cdf_mul(cdf a, cdf b) {
    return {df_dot2(a.x, b.x, df_neg(a.y), b.y), df_dot2(a.x, b.y, a.y, b.x)};
}
__device__ __forceinline__ cdf cdf_add(cdf a, cdf b) { return {df_add(a.x, b.x), df_add(a.y, b.y)}; }

// complex double-float product (non-template: preferred over the generic cx<R> operator)
__device__ __forceinline__ cx<df> operator*(cx<df> a, cx<df> b) {
    return mk<df>(df_dot2(a.x, b.x, df_neg(a.y), b.y), df_dot2(a.x, b.y, a.y, b.x));
}

// lazy double-float accumulator: leading sum with exact Knuth errors, all errors and low
// parts gathered in a float32 tail; value = hi + lo after the final renormalisation
struct dfacc {
    float hi, lo;
};
__device__ __forceinline__ void dfacc_add(dfacc& a, df v) {
    df s = df_two_sum(a.hi, v.hi);
    a.hi = s.hi;
    a.lo = __fadd_rn(a.lo, __fadd_rn(s.lo, v.lo));
}
__device__ __forceinline__ df dfacc_get(dfacc a) { return df_fast_sum(a.hi, a.lo); }
// a += x * y: Dekker's product (leading part exact by FMA) summed into the accumulator
// without renormalising the product first
__device__ __forceinline__ void dfacc_add_prod(dfacc& a, df x, df y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    const df s = df_two_sum(a.hi, p);
    a.hi = s.hi;
    a.lo = __fadd_rn(a.lo, __fadd_rn(s.lo, e));
}

constexpr int kCisTableBig = 1024;

// phase s . d in turns for df triples s and d: Dekker products with their exact FMA errors,
// Knuth sums of the leading parts, every small term gathered in float32, one renormalisation
__device__ __forceinline__ df df_dot3(const df* s, const df* d) {
    const float p0 = __fmul_rn(s[0].hi, d[0].hi), p1 = __fmul_rn(s[1].hi, d[1].hi), p2 = __fmul_rn(s[2].hi, d[2].hi);
    float e = __fadd_rn(__fadd_rn(__fmaf_rn(s[0].hi, d[0].hi, -p0), __fmaf_rn(s[1].hi, d[1].hi, -p1)),
                        __fmaf_rn(s[2].hi, d[2].hi, -p2));
    e = __fmaf_rn(s[0].hi, d[0].lo, __fmaf_rn(s[0].lo, d[0].hi, e));
    e = __fmaf_rn(s[1].hi, d[1].lo, __fmaf_rn(s[1].lo, d[1].hi, e));
    e = __fmaf_rn(s[2].hi, d[2].lo, __fmaf_rn(s[2].lo, d[2].hi, e));
    const df a = df_two_sum(p0, p1);
    const df b = df_two_sum(a.hi, p2);
    return df_fast_sum(b.hi, __fadd_rn(__fadd_rn(a.lo, b.lo), e));
}

// exp(2 pi i t) for any df t (turns): one reduction by the nearest 1/1024 of a turn (exact
// on the leading part), x = 2 pi r with |x| <= pi / 1024, then Taylor terms.  The result has
// modulus 1, so each term needs an absolute error below ~2^-49 only: x, x^2 and 1 - x^2/2
// are kept as double-float pairs (exact products by FMA, an exact Fast2Sum for 1 - x^2/2);
// x^4/24 (< 4e-12), x^3/6 (< 5e-9) and x^5/120 (< 3e-15) enter as float32 corrections of
// the low parts (rounding below 3e-16).  One fused complex product with the table entry.
__device__ __forceinline__ cdf cis_turns_big(df t, const cdf* tab) {
    const float jf = rintf(__fmul_rn(t.hi, (float)kCisTableBig));
    const df rr = df_fast_sum(__fsub_rn(t.hi, __fmul_rn(jf, 1.0f / (float)kCisTableBig)), t.lo);  // exact
    const df two_pi = {6.2831854820251465f, -1.7484555314695172e-07f};
    const df x = df_mul(rr, two_pi);
    // y = x^2 = yh + ye (|ye| small, not renormalised)
    const float yh = __fmul_rn(x.hi, x.hi);
    const float ye = __fmaf_rn(__fadd_rn(x.hi, x.hi), x.lo, __fmaf_rn(x.hi, x.hi, -yh));
    // cos x = 1 - y/2 + y^2/24: 1 - yh/2 exactly as (c, ce), the rest into the low part
    const float h = __fmul_rn(-0.5f, yh);
    const float c = __fadd_rn(1.0f, h);
    const float ce = __fsub_rn(h, __fsub_rn(c, 1.0f));
    const float clo = __fmaf_rn(__fmul_rn(yh, yh), 1.0f / 24.0f, __fmaf_rn(-0.5f, ye, ce));
    const df cc = df_fast_sum(c, clo);
    // sin x = x - x^3/6 + x^5/120: the two odd terms as one float32 correction
    const float x3 = __fmul_rn(x.hi, yh);
    const float corr = __fmul_rn(x3, __fmaf_rn(yh, 1.0f / 120.0f, -1.0f / 6.0f));
    const df ss = df_fast_sum(x.hi, __fadd_rn(x.lo, corr));
    const int j = ((int)jf) & (kCisTableBig - 1);
    return cdf_mul(tab[j], cdf{cc, ss});
}

}  // namespace hfmm
