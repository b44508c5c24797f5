// Double-float ("df") arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2, both float32,
// about 48 significant bits.  Built from error-free transformations: Knuth's TwoSum,
// Dekker's Fast2Sum and the FMA form of Dekker's exact product.  Every step uses the
// _rn intrinsics so the compiler cannot contract or reassociate it.
//
// cis_turns(r) = exp(2 pi i r) for |r| <= 1/2: reduction by a 256-entry table of
// exp(2 pi i j / 256) (stored as df pairs), then Taylor polynomials of sin and cos on
// |x| <= pi/256 in df arithmetic, then one complex df product.
#pragma once
#include <cuda_runtime.h>

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
__device__ __forceinline__ cdf cdf_mul(cdf a, cdf b) {
    return {df_sub(df_mul(a.x, b.x), df_mul(a.y, b.y)), df_add(df_mul(a.x, b.y), df_mul(a.y, b.x))};
}
__device__ __forceinline__ cdf cdf_add(cdf a, cdf b) { return {df_add(a.x, b.x), df_add(a.y, b.y)}; }

constexpr int kCisTable = 256;

// exp(2 pi i r) for |r| <= 1/2 (r in turns, as df); tab[j] = exp(2 pi i j / 256) as df pairs
__device__ __forceinline__ cdf cis_turns(df r, const cdf* tab) {
    const float jf = rintf(__fmul_rn(r.hi, (float)kCisTable));
    // r - j/256 is exact on the hi part (Sterbenz)
    df rr = df_fast_sum(__fsub_rn(r.hi, __fdiv_rn(jf, (float)kCisTable)), r.lo);
    const df two_pi = {6.2831854820251465f, -1.7484555314695172e-07f};
    df x = df_mul(rr, two_pi);                  // |x| <= pi / 256
    df y = df_mul(x, x);
    // cos x = 1 - y/2 + y^2/24 - y^3/720 ; sin x = x (1 - y/6 + y^2/120 - y^3/5040)
    const float yh = y.hi;
    const df c24 = {0.0416666679084301f, -1.2417634698280722e-09f};     // 1/24
    const df c6 = {0.1666666716337204f, -4.967053879312289e-09f};       // 1/6
    const df c120 = {0.008333333767950535f, -4.34617203337595e-10f};   // 1/120
    // every addition below has a dominant left operand (|y| <= 1.6e-4): Fast2Sum suffices
    df cc = df_add_big(c24, {__fmul_rn(yh, -1.0f / 720.0f), 0.0f});
    cc = df_mul(y, cc);
    cc = df_add_big({-0.5f, 0.0f}, cc);
    cc = df_mul(y, cc);
    cc = df_add_big({1.0f, 0.0f}, cc);
    df ss = df_add_big(c120, {__fmul_rn(yh, -1.0f / 5040.0f), 0.0f});
    ss = df_mul(y, ss);
    ss = df_add_big(df_neg(c6), ss);
    ss = df_mul(y, ss);
    ss = df_mul(x, ss);
    ss = df_add_big(x, ss);
    const int j = ((int)jf) & (kCisTable - 1);
    return cdf_mul(tab[j], cdf{cc, ss});
}

}  // namespace hfmm
