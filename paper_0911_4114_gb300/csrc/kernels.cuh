// Stage kernels of the FMM apply (Section 2 of the paper on the Section 3 quadratures).
// Signatures are stored box-major: sig[(box * R + r) * K + k], k over the half grid
// (rows n = 0..ntheta/2, N_phi(theta_n) samples each).
#pragma once
#include <type_traits>

#include "cx.cuh"
#include "df.cuh"
#include "fft.cuh"

namespace hfmm {

constexpr int kWarps = 4;  // warps per CTA in the re-sampling kernels

struct QuadView {
    int ntheta;        // even
    int nrows;         // ntheta / 2 + 1
    int64_t K;
    const int* nphi;   // nrows
    const int64_t* off;  // nrows + 1
    const double* shat;  // (K, 3)
    const double* w;     // (K) folded quadrature weights
    // antipodal pairs (k, k'): s_k' = -s_k, so exp(i k s_k' . d) = conj(exp(i k s_k . d)).
    // Row n mirrors row N_theta/2 - n with the same N_phi (a multiple of 4), so sample
    // (n, m) pairs with (N_theta/2 - n, m + N_phi/2); npair = K / 2.
    const int2* pair;
    int64_t npair;
    // (K, 6) floats per sample: kappa s_k / (2 pi) split into a leading float and the float
    // rounding of the rest (hi x, y, z, lo x, y, z): float32 levels form plane-wave phases
    // from these without float64 arithmetic
    const float* asplit;
};

struct BoxView {
    int nbox;
    const double* center;      // (nbox, 3)
    const int32_t* idx;        // (nbox, 3)
    const int32_t* parent;
    const int32_t* child_start;
    const int32_t* child_count;
    // S2M / L2T / far gradient of an adaptive tree: block x works on box leaf[x] (the level's
    // leaves); null: on box x
    const int32_t* leaf = nullptr;
};

// ---------------------------------------------------------------------------
// permutations
// ---------------------------------------------------------------------------
template <typename Tin, bool kConj>
__global__ void k_permute_in(const cx<Tin>* __restrict__ q, int64_t n, int R,
                             const int64_t* __restrict__ perm, cxd* __restrict__ qs) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * R) return;
    int64_t p = t / R;
    int r = (int)(t - p * R);
    cxd v = cvt<double>(q[perm[p] * R + r]);
    qs[t] = kConj ? conj(v) : v;
}

template <typename Tout, bool kConj>
__global__ void k_permute_out(const cxd* __restrict__ phis, int64_t n, int R,
                              const int64_t* __restrict__ perm, cx<Tout>* __restrict__ phi) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * R) return;
    int64_t p = t / R;
    int r = (int)(t - p * R);
    cxd v = kConj ? conj(phis[t]) : phis[t];
    phi[perm[p] * R + r] = cvt<Tout>(v);
}

// ---------------------------------------------------------------------------
// near field (P2P), float64: phi_i = sum_{j in N(b), R > 0} q_j exp(i k R) / R
// one CTA per target leaf box, sources staged through shared memory
// ---------------------------------------------------------------------------
constexpr int kP2PThreads = 128;
constexpr int kP2PTile = 128;      // sources staged per barrier (mixed near field): one float32 tile sum

__global__ void k_p2p_fp64(int nbox, const int32_t* __restrict__ tstart, const int32_t* __restrict__ tcount,
                           const int32_t* __restrict__ sstart, const int32_t* __restrict__ scount,
                           const int32_t* __restrict__ noff, const int32_t* __restrict__ nidx,
                           const double* __restrict__ tx, const double* __restrict__ ty,
                           const double* __restrict__ tz, const double* __restrict__ sx,
                           const double* __restrict__ sy, const double* __restrict__ sz,
                           const cxd* __restrict__ qs, cxd* __restrict__ phis, int R, double kappa) {
    __shared__ double shx[kP2PThreads], shy[kP2PThreads], shz[kP2PThreads];
    __shared__ cxd shq[kP2PThreads * 4];
    const int b = blockIdx.x;
    if (b >= nbox) return;
    const int t0 = tstart[b], tc = tcount[b];
    if ((int)blockIdx.y * kP2PThreads >= tc) return;
    for (int r0 = 0; r0 < R; r0 += 4) {
        const int rn = min(4, R - r0);
        {
            const int tb = blockIdx.y * kP2PThreads;
            const int ti = tb + threadIdx.x;
            const bool active = ti < tc;
            double x = 0, y = 0, z = 0;
            if (active) {
                x = tx[t0 + ti];
                y = ty[t0 + ti];
                z = tz[t0 + ti];
            }
            cxd acc[4];
            for (int r = 0; r < 4; ++r) acc[r] = mk<double>(0, 0);
            for (int nb = noff[b]; nb < noff[b + 1]; ++nb) {
                const int s = nidx[nb];
                const int s0 = sstart[s], sc = scount[s];
                for (int sb = 0; sb < sc; sb += kP2PThreads) {
                    const int sn = min(kP2PThreads, sc - sb);
                    __syncthreads();
                    if (threadIdx.x < sn) {
                        const int j = s0 + sb + threadIdx.x;
                        shx[threadIdx.x] = sx[j];
                        shy[threadIdx.x] = sy[j];
                        shz[threadIdx.x] = sz[j];
                        for (int r = 0; r < rn; ++r) shq[threadIdx.x * 4 + r] = qs[(int64_t)j * R + r0 + r];
                    }
                    __syncthreads();
                    if (active) {
                        for (int jj = 0; jj < sn; ++jj) {
                            const double dx = x - shx[jj], dy = y - shy[jj], dz = z - shz[jj];
                            const double r2 = dx * dx + dy * dy + dz * dz;
                            if (r2 == 0.0) continue;
                            const double rr = sqrt(r2);
                            double sn_, cs_;
                            sincos(kappa * rr, &sn_, &cs_);
                            const double inv = 1.0 / rr;
                            const cxd g = mk<double>(cs_ * inv, sn_ * inv);
                            for (int r = 0; r < rn; ++r) mac(acc[r], g, shq[jj * 4 + r]);
                        }
                    }
                }
            }
            if (active)
                for (int r = 0; r < rn; ++r) phis[(int64_t)(t0 + ti) * R + r0 + r] = acc[r];
        }
    }
}

// ---------------------------------------------------------------------------
// near field, mixed precision: float32 arithmetic on exactly representable grid
// coordinates (integer part g on a 2^12 grid of the root cube, fractional part o in
// [0,1)), squared distance kept as (A exact, B small) and one Newton step on the
// square root, phase reduced in turns with a split constant; float64 accumulation of
// float32 tile sums.
// ---------------------------------------------------------------------------
// hardware approximations without subnormal handling, for arguments that are zero or normal:
// reciprocal square root, and sine and cosine of |x| <= pi (the approximations that rsqrtf
// and __sincosf reach after their subnormal checks, which these arguments never need)
__device__ __forceinline__ float rsqrt_hw(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ void sincos_hw(float x, float* s, float* c) {
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(*s) : "f"(x));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(*c) : "f"(x));
}

struct P2PMixedArgs {
    const float4* tpt;   // (gx, gy, gz, 0) per sorted target
    const float4* tof;   // (ox, oy, oz, 0)
    const float4* spt;
    const float4* sof;
    float tau_hi, tau_lo;  // turns per grid unit (kappa * side / 2^12 / 2 pi), split
    double inv_unit;       // 2^12 / side: 1 / (grid unit in length)
    float inv_unit_f;
};

// float -> double by assembling the bits (exact for normal numbers and zero; subnormal
// floats become zero), keeping the conversion off the slow float64 pipe
__device__ __forceinline__ double f2d_bits(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t sign = u & 0x80000000u, ex = (u >> 23) & 0xffu, man = u & 0x7fffffu;
    if (ex == 0) return __hiloint2double((int)sign, 0);
    return __hiloint2double((int)(sign | ((ex + 896u) << 20) | (man >> 3)), (int)(man << 29));
}

// ---------------------------------------------------------------------------
// S2M: M_b(s_k) = sum_{j in b} q_j exp(i k s_k . (y_j - c_b)) at the leaf level
// thread per (box, k); sources of the box staged through shared memory
// ---------------------------------------------------------------------------
constexpr int kS2MThreads = 128;
constexpr int kS2MTile = 256;      // sources staged per barrier (double-float S2M)

template <typename R>
__device__ __forceinline__ cx<R> plane_wave(double phase_turns_reduced);

template <>
__device__ __forceinline__ cxd plane_wave<double>(double t) {
    double s, c;
    sincospi(2.0 * t, &s, &c);
    return mk<double>(c, s);
}
template <>
__device__ __forceinline__ cxf plane_wave<float>(double t) {
    float s, c;
    sincospif(2.0f * (float)t, &s, &c);
    return mk<float>(c, s);
}

// phase kappa * (s . d) in turns, reduced to [-1/2, 1/2]
__device__ __forceinline__ double turns(double kappa_turns, const double* s, double dx, double dy, double dz) {
    double p = kappa_turns * (s[0] * dx + s[1] * dy + s[2] * dz);
    return p - rint(p);
}

// The same reduced phase in float32 arithmetic only, for float32 levels (float64 runs at 1/64
// of the float32 rate on this GPU).  a = kappa s / (2 pi) and d are given as float pairs
// (hi, lo), each exact to about 2^-48.  The leading products a_hi d_hi are formed exactly (FMA
// error terms) and summed with Knuth's TwoSum, so the integer part drops out exactly
// (s - rint(s) is exact in float); the error terms and the cross products a_hi d_lo, a_lo d_hi
// are added to the reduced fraction.  Absolute error about 2^-25 turns, the size of the
// rounding of a float64 phase reduced into [-1/2, 1/2] and converted to float.
__device__ __forceinline__ float two_sum_err(float a, float b, float s) {
    const float bb = s - a;
    return (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ float turns_f(const float* a, const float* d) {
    const float p0 = a[0] * d[0], p1 = a[1] * d[1], p2 = a[2] * d[2];
    const float e0 = fmaf(a[0], d[0], -p0), e1 = fmaf(a[1], d[1], -p1), e2 = fmaf(a[2], d[2], -p2);
    const float s1 = p0 + p1;
    const float s2 = s1 + p2;
    const float err = two_sum_err(p0, p1, s1) + two_sum_err(s1, p2, s2);
    const float cross = fmaf(a[0], d[3], fmaf(a[1], d[4], fmaf(a[2], d[5], fmaf(a[3], d[0], fmaf(a[4], d[1], a[5] * d[2])))));
    return (s2 - rintf(s2)) + ((err + (e0 + e1 + e2)) + cross);
}
__device__ __forceinline__ void split_f(double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

// Points to signature: M_b(s_k) = w_k sum_{j in b} exp(i k s_k . sign (p_j - c_b)) q_j.
// S2M: sources, sign +1, no weights.  Transposed L2T: targets, sign -1, quadrature weights.
// One thread per antipodal pair (k, k'): with E = C + iS the plane wave of s_k, it sums
// U = sum q C and V = sum q S; then M(k) = U + iV and M(k') = U - iV.  kRC right-hand
// sides per plane-wave evaluation (1, 4, or 16 at float32 levels with many right-hand
// sides).  The charges are rounded to the level's precision once, as they enter shared
// memory (a float64 -> float32 conversion per use would run on the slow float64 pipe).
template <typename R, int kRC>
__global__ void k_s2m(BoxView bx, QuadView qv, const int32_t* __restrict__ sstart,
                      const int32_t* __restrict__ scount, const double* __restrict__ sx,
                      const double* __restrict__ sy, const double* __restrict__ sz,
                      const cxd* __restrict__ qs, int R_, double kappa_turns, cx<R>* __restrict__ M,
                      double sign, const double* __restrict__ wk) {
    constexpr bool kF32 = std::is_same<R, float>::value;   // float32 level: float-only phases
    __shared__ double shd[kS2MThreads * 3];
    __shared__ float shf[kS2MThreads * 6];
    __shared__ cx<R> shq[kS2MThreads * kRC];
    const int b = bx.leaf ? bx.leaf[blockIdx.x] : (int)blockIdx.x;
    const int64_t p = blockIdx.y * (int64_t)blockDim.x + threadIdx.x;
    const bool active = p < qv.npair;
    int2 kk2 = make_int2(0, 0);
    double s[3] = {0, 0, 0};
    float af[6] = {0, 0, 0, 0, 0, 0};
    if (active) {
        kk2 = qv.pair[p];
        s[0] = qv.shat[3 * kk2.x];
        s[1] = qv.shat[3 * kk2.x + 1];
        s[2] = qv.shat[3 * kk2.x + 2];
        if (kF32)
            for (int c = 0; c < 6; ++c) af[c] = qv.asplit[6 * (int64_t)kk2.x + c];
    }
    const int s0 = sstart[b], sc = scount[b];
    const double cxx = bx.center[3 * b], cyy = bx.center[3 * b + 1], czz = bx.center[3 * b + 2];
    for (int r0 = 0; r0 < R_; r0 += kRC) {
        const int rn = kRC == 1 ? 1 : min(kRC, R_ - r0);
        cx<R> U[kRC], V[kRC];
        for (int r = 0; r < kRC; ++r) U[r] = V[r] = mk<R>(0, 0);
        for (int jb = 0; jb < sc; jb += kS2MThreads) {
            const int jn = min(kS2MThreads, sc - jb);
            __syncthreads();
            if (threadIdx.x < jn) {
                const int j = s0 + jb + threadIdx.x;
                const double dd[3] = {sign * (sx[j] - cxx), sign * (sy[j] - cyy), sign * (sz[j] - czz)};
                for (int c = 0; c < 3; ++c) {
                    shd[3 * threadIdx.x + c] = dd[c];
                    split_f(dd[c], shf[6 * threadIdx.x + c], shf[6 * threadIdx.x + 3 + c]);
                }
                for (int r = 0; r < rn; ++r) shq[threadIdx.x * kRC + r] = cvt<R>(qs[(int64_t)j * R_ + r0 + r]);
            }
            __syncthreads();
            if (active)
                for (int jj = 0; jj < jn; ++jj) {
                    cx<R> e;
                    if (kF32) {
                        float sn, cs;
                        sincospif(2.0f * turns_f(af, &shf[6 * jj]), &sn, &cs);
                        e = mk<R>(cs, sn);
                    } else {
                        e = plane_wave<R>(turns(kappa_turns, s, shd[3 * jj], shd[3 * jj + 1], shd[3 * jj + 2]));
                    }
#pragma unroll
                    for (int r = 0; r < kRC; ++r)
                        if (r < rn) {
                            const cx<R> q = shq[jj * kRC + r];
                            U[r] = U[r] + e.x * q;
                            V[r] = V[r] + e.y * q;
                        }
                }
        }
        if (active)
#pragma unroll
            for (int r = 0; r < kRC; ++r) {
                if (r >= rn) break;
                cx<R> a = mk<R>(U[r].x - V[r].y, U[r].y + V[r].x), c = mk<R>(U[r].x + V[r].y, U[r].y - V[r].x);
                if (wk) {
                    a = (R)wk[kk2.x] * a;
                    c = (R)wk[kk2.y] * c;
                }
                M[((int64_t)b * R_ + r0 + r) * qv.K + kk2.x] = a;
                M[((int64_t)b * R_ + r0 + r) * qv.K + kk2.y] = c;
            }
    }
}

// ---------------------------------------------------------------------------
// L2T: phi_i += sum_k w_k L_b(s_k) exp(i k s_k . (c_b - x_i)); thread per target
// ---------------------------------------------------------------------------
constexpr int kL2TThreads = 128;

// Signature to points: phi_i += sum_k w_k L_b(s_k) exp(i k s_k . sign (c_b - p_i)).
// L2T: targets, sign +1, quadrature weights.  Transposed S2M: sources, sign -1, no weights.
// Over antipodal pairs (k, k') with A = w_k L(k), B = w_k' L(k'), E = C + iS the plane wave
// of s_k: A E + B conj(E) = (P.x C - Q.y S) + i (P.y C + Q.x S), P = A + B, Q = A - B.
// kRC right-hand sides per plane-wave evaluation (1, 4, or 16 at float32 levels with many
// right-hand sides).
template <typename R, int kRC>
__global__ void k_l2t(BoxView bx, QuadView qv, const int32_t* __restrict__ tstart,
                      const int32_t* __restrict__ tcount, const double* __restrict__ tx,
                      const double* __restrict__ ty, const double* __restrict__ tz,
                      const cx<R>* __restrict__ L, int R_, double kappa_turns, cxd* __restrict__ phis,
                      double sign, const double* __restrict__ wk) {
    constexpr bool kF32 = std::is_same<R, float>::value;   // float32 level: float-only phases
    __shared__ double shs[kL2TThreads * 3];
    __shared__ float shf[kL2TThreads * 6];
    __shared__ cx<R> shp[kL2TThreads * kRC], shq[kL2TThreads * kRC];
    const int b = bx.leaf ? bx.leaf[blockIdx.x] : (int)blockIdx.x;
    const int t0 = tstart[b], tc = tcount[b];
    if ((int)blockIdx.y * kL2TThreads >= tc) return;
    const double cxx = bx.center[3 * b], cyy = bx.center[3 * b + 1], czz = bx.center[3 * b + 2];
    const int ti = blockIdx.y * kL2TThreads + threadIdx.x;
    const bool active = ti < tc;
    double dx = 0, dy = 0, dz = 0;
    float df6[6] = {0, 0, 0, 0, 0, 0};
    if (active) {
        dx = sign * (cxx - tx[t0 + ti]);
        dy = sign * (cyy - ty[t0 + ti]);
        dz = sign * (czz - tz[t0 + ti]);
        split_f(dx, df6[0], df6[3]);
        split_f(dy, df6[1], df6[4]);
        split_f(dz, df6[2], df6[5]);
    }
    for (int r0 = 0; r0 < R_; r0 += kRC) {
        const int rn = kRC == 1 ? 1 : min(kRC, R_ - r0);
        cx<R> acc[kRC];
        for (int r = 0; r < kRC; ++r) acc[r] = mk<R>(0, 0);
        for (int64_t pb = 0; pb < qv.npair; pb += kL2TThreads) {
            const int pn = (int)min((int64_t)kL2TThreads, qv.npair - pb);
            __syncthreads();
            if (threadIdx.x < pn) {
                const int2 kk2 = qv.pair[pb + threadIdx.x];
                shs[3 * threadIdx.x] = qv.shat[3 * kk2.x];
                shs[3 * threadIdx.x + 1] = qv.shat[3 * kk2.x + 1];
                shs[3 * threadIdx.x + 2] = qv.shat[3 * kk2.x + 2];
                if (kF32)
                    for (int c = 0; c < 6; ++c) shf[6 * threadIdx.x + c] = qv.asplit[6 * (int64_t)kk2.x + c];
                for (int r = 0; r < rn; ++r) {
                    const cx<R>* Lb = L + ((int64_t)b * R_ + r0 + r) * qv.K;
                    const cx<R> A = wk ? (R)wk[kk2.x] * Lb[kk2.x] : Lb[kk2.x];
                    const cx<R> B = wk ? (R)wk[kk2.y] * Lb[kk2.y] : Lb[kk2.y];
                    shp[threadIdx.x * kRC + r] = A + B;
                    shq[threadIdx.x * kRC + r] = A - B;
                }
            }
            __syncthreads();
            if (active)
                for (int kk = 0; kk < pn; ++kk) {
                    cx<R> e;
                    if (kF32) {
                        float sn, cs;
                        sincospif(2.0f * turns_f(&shf[6 * kk], df6), &sn, &cs);
                        e = mk<R>(cs, sn);
                    } else {
                        e = plane_wave<R>(turns(kappa_turns, &shs[3 * kk], dx, dy, dz));
                    }
#pragma unroll
                    for (int r = 0; r < kRC; ++r)
                        if (r < rn) {
                            const cx<R> P = shp[kk * kRC + r], Q = shq[kk * kRC + r];
                            acc[r].x += P.x * e.x - Q.y * e.y;
                            acc[r].y += P.y * e.x + Q.x * e.y;
                        }
                }
        }
        if (active)
#pragma unroll
            for (int r = 0; r < kRC; ++r) {
                if (r >= rn) break;
                cxd& o = phis[(int64_t)(t0 + ti) * R_ + r0 + r];
                o.x += (double)acc[r].x;
                o.y += (double)acc[r].y;
            }
    }
}

// ---------------------------------------------------------------------------
// Plane-wave tables of a float64 leaf level.  GB300 executes float64 at 1/64 of the float32
// rate: a float64 plane wave exp(i kappa s_k . (p - c_b)) (phase, reduction, sincospi) costs
// tens of float64 operations, the sums that use it 4 FMA per right-hand side.  The plan
// therefore evaluates every plane wave of the leaf level once into HBM,
//     E[j][p] = exp(i kappa s_k . (p_j - c_b)),  k = pair[p].x,
// for every sorted point j (leaf box b) and antipodal pair p, with the same arithmetic as
// k_s2m (phase in turns, reduced, sincospi), and S2M / L2T and their transposes read it:
// one 16-byte load and 4 FMA per (point, pair, RHS).  The plane wave of s_k' = -s_k is the
// conjugate, and the opposite offset (c_b - p_j) conjugates too.
// ---------------------------------------------------------------------------
constexpr int kTabThreads = 128;

// one block per (leaf box, 32-point chunk) x 128 pairs; E row-major [point][pair]
__global__ void __launch_bounds__(kTabThreads) k_pw_table(
    const int2* __restrict__ units, BoxView bx, QuadView qv, const int32_t* __restrict__ pstart,
    const int32_t* __restrict__ pcount, const double* __restrict__ px, const double* __restrict__ py,
    const double* __restrict__ pz, double kappa_turns, cxd* __restrict__ E) {
    const int b = units[blockIdx.x].x, c0 = units[blockIdx.x].y;
    const int64_t p = blockIdx.y * (int64_t)kTabThreads + threadIdx.x;
    if (p >= qv.npair) return;
    const int k = qv.pair[p].x;
    const double s[3] = {qv.shat[3 * k], qv.shat[3 * k + 1], qv.shat[3 * k + 2]};
    const double cxx = bx.center[3 * b], cyy = bx.center[3 * b + 1], czz = bx.center[3 * b + 2];
    const int n = min(32, pcount[b] - c0);
    for (int jj = 0; jj < n; ++jj) {
        const int64_t j = pstart[b] + c0 + jj;
        const double t = turns(kappa_turns, s, px[j] - cxx, py[j] - cyy, pz[j] - czz);
        E[j * qv.npair + p] = plane_wave<double>(t);
    }
}

// points -> signature from the table (S2M: sources, E as stored; transposed L2T: targets,
// conjugated, weighted).  Thread per (box, antipodal pair); U = sum q C, V = sum q S over the
// box's points, M(k) = U + iV, M(k') = U - iV (as k_s2m).  kRC right-hand sides per pass.
template <int kRC, bool kConj>
__global__ void __launch_bounds__(kTabThreads) k_s2m_tab(
    QuadView qv, const int32_t* __restrict__ sstart, const int32_t* __restrict__ scount,
    const cxd* __restrict__ E, const cxd* __restrict__ qs, int R_, cxd* __restrict__ M,
    const double* __restrict__ wk) {
    const int b = blockIdx.x;
    const int64_t p = blockIdx.y * (int64_t)kTabThreads + threadIdx.x;
    if (p >= qv.npair) return;
    const int2 kk2 = qv.pair[p];
    const int s0 = sstart[b], sc = scount[b];
    const cxd* Ep = E + (int64_t)s0 * qv.npair + p;
    for (int r0 = 0; r0 < R_; r0 += kRC) {
        const int rn = kRC == 1 ? 1 : min(kRC, R_ - r0);
        cxd U[kRC], V[kRC];
        for (int r = 0; r < kRC; ++r) U[r] = V[r] = mk<double>(0, 0);
        for (int jj = 0; jj < sc; ++jj) {
            cxd e = ldg_cx(Ep + (int64_t)jj * qv.npair);
            if (kConj) e.y = -e.y;
            const cxd* qj = qs + (int64_t)(s0 + jj) * R_ + r0;
            for (int r = 0; r < rn; ++r) {
                const cxd q = ldg_cx(qj + r);
                U[r] = U[r] + e.x * q;
                V[r] = V[r] + e.y * q;
            }
        }
        for (int r = 0; r < rn; ++r) {
            cxd a = mk<double>(U[r].x - V[r].y, U[r].y + V[r].x), c = mk<double>(U[r].x + V[r].y, U[r].y - V[r].x);
            if (wk) {
                a = wk[kk2.x] * a;
                c = wk[kk2.y] * c;
            }
            M[((int64_t)b * R_ + r0 + r) * qv.K + kk2.x] = a;
            M[((int64_t)b * R_ + r0 + r) * qv.K + kk2.y] = c;
        }
    }
}

// signature -> points from the table (L2T: targets, conjugated, weighted; transposed S2M:
// sources, E as stored).  One block per (leaf box, 32-point chunk); warp w takes points
// w, w + 8, w + 16, w + 24 of the chunk, its lanes stride the antipodal pairs (coalesced
// table rows); P = A + B, Q = A - B (A = w_k L(k), B = w_k' L(k')) are staged in shared
// memory 128 pairs at a time; A E + B conj(E) = (P.x C - Q.y S) + i (P.y C + Q.x S).
constexpr int kL2TabWarps = 8;
constexpr int kL2TabChunk = 128;

template <int kRC, bool kConj>
__global__ void __launch_bounds__(32 * kL2TabWarps) k_l2t_tab(
    const int2* __restrict__ units, QuadView qv, const int32_t* __restrict__ pstart,
    const int32_t* __restrict__ pcount, const cxd* __restrict__ E, const cxd* __restrict__ L, int R_,
    cxd* __restrict__ out, const double* __restrict__ wk) {
    constexpr int kPts = 32 / kL2TabWarps;
    __shared__ cxd shp[kL2TabChunk * kRC], shq[kL2TabChunk * kRC];
    const int b = units[blockIdx.x].x, c0 = units[blockIdx.x].y;
    const int t0 = pstart[b], n = min(32, pcount[b] - c0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r0 = 0; r0 < R_; r0 += kRC) {
        const int rn = kRC == 1 ? 1 : min(kRC, R_ - r0);
        cxd acc[kPts][kRC];
        for (int i = 0; i < kPts; ++i)
            for (int r = 0; r < kRC; ++r) acc[i][r] = mk<double>(0, 0);
        for (int64_t pb = 0; pb < qv.npair; pb += kL2TabChunk) {
            const int pn = (int)min((int64_t)kL2TabChunk, qv.npair - pb);
            __syncthreads();
            for (int v = threadIdx.x; v < pn * kRC; v += blockDim.x) {
                const int pp = v / kRC, r = v % kRC;
                cxd P = mk<double>(0, 0), Q = P;
                if (r < rn) {
                    const int2 kk2 = qv.pair[pb + pp];
                    const cxd* Lb = L + ((int64_t)b * R_ + r0 + r) * qv.K;
                    const cxd A = wk ? wk[kk2.x] * Lb[kk2.x] : Lb[kk2.x];
                    const cxd B = wk ? wk[kk2.y] * Lb[kk2.y] : Lb[kk2.y];
                    P = A + B;
                    Q = A - B;
                }
                shp[pp * kRC + r] = P;
                shq[pp * kRC + r] = Q;
            }
            __syncthreads();
            // the warp's points side by side: kPts independent table loads in flight per lane,
            // and each staged P, Q serves all of them (points past the chunk read nothing and
            // add zeros)
#pragma unroll 2
            for (int pp = lane; pp < pn; pp += 32) {
                cxd e[kPts];
#pragma unroll
                for (int i = 0; i < kPts; ++i) {
                    const int ti = warp + kL2TabWarps * i;
                    e[i] = ti < n ? ldg_cx(E + (int64_t)(t0 + c0 + ti) * qv.npair + pb + pp) : mk<double>(0, 0);
                    if (kConj) e[i].y = -e[i].y;
                }
                for (int r = 0; r < rn; ++r) {
                    const cxd P = shp[pp * kRC + r], Q = shq[pp * kRC + r];
#pragma unroll
                    for (int i = 0; i < kPts; ++i) {   // four FMA, no separate product or sum
                        acc[i][r].x = fma(P.x, e[i].x, fma(-Q.y, e[i].y, acc[i][r].x));
                        acc[i][r].y = fma(P.y, e[i].x, fma(Q.x, e[i].y, acc[i][r].y));
                    }
                }
            }
        }
        for (int i = 0; i < kPts; ++i) {
            const int ti = warp + kL2TabWarps * i;
            if (ti >= n) break;
            for (int r = 0; r < rn; ++r) {
                double x = acc[i][r].x, y = acc[i][r].y;
                for (int o = 16; o > 0; o >>= 1) {
                    x += __shfl_xor_sync(0xffffffffu, x, o);
                    y += __shfl_xor_sync(0xffffffffu, y, o);
                }
                if (lane == 0) {
                    cxd& o = out[(int64_t)(t0 + c0 + ti) * R_ + r0 + r];
                    o.x += x;
                    o.y += y;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// S2M and L2T of float64 levels in double-float arithmetic on the float32 pipe (about 48
// significant bits; float64 in memory).  s' = s_k * kappa / (2 pi) and the offsets are
// split into df pairs; the phase in turns is reduced by its nearest integer and cis_turns
// evaluates exp(2 pi i r).
// ---------------------------------------------------------------------------
// kRC right-hand sides per plane-wave evaluation (1, or 4 when R > 1).
template <int kRC>
__global__ void k_s2m_df(BoxView bx, QuadView qv, const int32_t* __restrict__ sstart,
                         const int32_t* __restrict__ scount, const double* __restrict__ sx,
                         const double* __restrict__ sy, const double* __restrict__ sz,
                         const cxd* __restrict__ qs, int R_, double kappa_turns, const cdf* __restrict__ cis_tab,
                         cx<df>* __restrict__ M, double sign, const double* __restrict__ wk) {
    __shared__ df shd[kS2MTile * 3];
    __shared__ cdf shq[kS2MTile * kRC];
    __shared__ cdf tab[kCisTableBig];
    for (int v = threadIdx.x; v < kCisTableBig; v += blockDim.x) tab[v] = cis_tab[v];
    const int b = bx.leaf ? bx.leaf[blockIdx.x] : (int)blockIdx.x;
    const int64_t p = blockIdx.y * (int64_t)blockDim.x + threadIdx.x;   // antipodal pair
    const bool active = p < qv.npair;
    int2 kk2 = make_int2(0, 0);
    df s[3] = {{0, 0}, {0, 0}, {0, 0}};
    if (active) {
        kk2 = qv.pair[p];
        for (int c = 0; c < 3; ++c) s[c] = df_from_double(qv.shat[3 * kk2.x + c] * kappa_turns);
    }
    const int s0 = sstart[b], sc = scount[b];
    const double cxx = bx.center[3 * b], cyy = bx.center[3 * b + 1], czz = bx.center[3 * b + 2];
    for (int r0 = 0; r0 < R_; r0 += kRC) {
        const int rn = kRC == 1 ? 1 : min(kRC, R_ - r0);
        // U = sum q C, V = sum q S with C + iS = exp(i k s_k . d)
        dfacc ux[kRC], uy[kRC], vx[kRC], vy[kRC];
        for (int r = 0; r < kRC; ++r) ux[r] = uy[r] = vx[r] = vy[r] = dfacc{0.f, 0.f};
        for (int jb = 0; jb < sc; jb += kS2MTile) {
            const int jn = min(kS2MTile, sc - jb);
            __syncthreads();
            for (int u = threadIdx.x; u < jn; u += kS2MThreads) {
                const int j = s0 + jb + u;
                shd[3 * u] = df_from_double(sign * (sx[j] - cxx));
                shd[3 * u + 1] = df_from_double(sign * (sy[j] - cyy));
                shd[3 * u + 2] = df_from_double(sign * (sz[j] - czz));
                for (int r = 0; r < rn; ++r) {
                    const cxd qq = qs[(int64_t)j * R_ + r0 + r];
                    shq[u * kRC + r] = cdf{df_from_double(qq.x), df_from_double(qq.y)};
                }
            }
            __syncthreads();
            if (active)
                for (int jj = 0; jj < jn; ++jj) {
                    const cdf e = cis_turns_big(df_dot3(s, &shd[3 * jj]), tab);
                    for (int r = 0; r < rn; ++r) {
                        const cdf q = shq[jj * kRC + r];
                        dfacc_add_prod(ux[r], q.x, e.x);
                        dfacc_add_prod(uy[r], q.y, e.x);
                        dfacc_add_prod(vx[r], q.x, e.y);
                        dfacc_add_prod(vy[r], q.y, e.y);
                    }
                }
        }
        if (active)
            for (int r = 0; r < rn; ++r) {
                const df Ux = dfacc_get(ux[r]), Uy = dfacc_get(uy[r]), Vx = dfacc_get(vx[r]), Vy = dfacc_get(vy[r]);
                cdf a = {df_sub(Ux, Vy), df_add(Uy, Vx)};   // M(k)  = U + iV
                cdf c = {df_add(Ux, Vy), df_sub(Uy, Vx)};   // M(k') = U - iV
                if (wk) {
                    const df wa = df_from_double(wk[kk2.x]), wc = df_from_double(wk[kk2.y]);
                    a = cdf{df_mul(a.x, wa), df_mul(a.y, wa)};
                    c = cdf{df_mul(c.x, wc), df_mul(c.y, wc)};
                }
                M[((int64_t)b * R_ + r0 + r) * qv.K + kk2.x] = mk<df>(a.x, a.y);
                M[((int64_t)b * R_ + r0 + r) * qv.K + kk2.y] = mk<df>(c.x, c.y);
            }
    }
}

// ---------------------------------------------------------------------------
// Warp-granular versions: one warp per (leaf box, 32-point chunk) work unit, warp-private
// shared staging and __syncwarp only, so a box's last partial chunk idles at most one warp
// and no warp waits at a block barrier for another box's work.
// ---------------------------------------------------------------------------
constexpr int kWarpTile = 64;    // quadrature samples (or sources) staged per warp step

// signature -> points, double-float (L2T: targets, sign +1, weights; transposed S2M: sources,
// sign -1, no weights); sdf = s_k * kappa / 2 pi as df triples, precomputed per level.
// kRC right-hand sides per plane-wave evaluation.
template <int kRC>
__global__ void __launch_bounds__(128) k_l2t_df_warp(
    const int2* __restrict__ units, int nunits, BoxView bx, QuadView qv, const df* __restrict__ sdf,
    const int32_t* __restrict__ pstart, const int32_t* __restrict__ pcount, const double* __restrict__ px,
    const double* __restrict__ py, const double* __restrict__ pz, const cx<df>* __restrict__ L, int R_,
    const cdf* __restrict__ cis_tab, cxd* __restrict__ out, double sign, const double* __restrict__ wk) {
    constexpr int kTile = kRC == 1 ? kWarpTile : 16;   // pairs staged per warp step
    __shared__ cdf tab[kCisTableBig];
    __shared__ df shs[4][kTile * 3];
    __shared__ cdf shp[4][kTile * kRC], shiq[4][kTile * kRC];
    for (int v = threadIdx.x; v < kCisTableBig; v += blockDim.x) tab[v] = cis_tab[v];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int u = blockIdx.x * 4 + warp;
    if (u >= nunits) return;
    const int b = units[u].x, c0 = units[u].y;
    const int t0 = pstart[b], tc = pcount[b];
    const int ti = c0 + lane;
    const bool active = ti < tc;
    const double cxx = bx.center[3 * b], cyy = bx.center[3 * b + 1], czz = bx.center[3 * b + 2];
    df d[3] = {{0, 0}, {0, 0}, {0, 0}};
    if (active) {
        d[0] = df_from_double(sign * (cxx - px[t0 + ti]));
        d[1] = df_from_double(sign * (cyy - py[t0 + ti]));
        d[2] = df_from_double(sign * (czz - pz[t0 + ti]));
    }
    df* ss = shs[warp];
    cdf* sp = shp[warp];
    cdf* siq = shiq[warp];
    for (int r0 = 0; r0 < R_; r0 += kRC) {
        const int rn = kRC == 1 ? 1 : min(kRC, R_ - r0);
        dfacc ax[kRC], ay[kRC];
        for (int r = 0; r < kRC; ++r) ax[r] = ay[r] = dfacc{0.f, 0.f};
        for (int64_t pb = 0; pb < qv.npair; pb += kTile) {
            const int pn = (int)min((int64_t)kTile, qv.npair - pb);
            __syncwarp();
            for (int v = lane; v < pn; v += 32) {
                const int2 kk2 = qv.pair[pb + v];
                ss[3 * v] = sdf[3 * kk2.x];
                ss[3 * v + 1] = sdf[3 * kk2.x + 1];
                ss[3 * v + 2] = sdf[3 * kk2.x + 2];
                df wa = {1.f, 0.f}, wb = {1.f, 0.f};
                if (wk) {
                    wa = df_from_double(wk[kk2.x]);
                    wb = df_from_double(wk[kk2.y]);
                }
                for (int r = 0; r < rn; ++r) {
                    const cx<df>* Lb = L + ((int64_t)b * R_ + r0 + r) * qv.K;
                    cdf A = cdf{Lb[kk2.x].x, Lb[kk2.x].y}, B = cdf{Lb[kk2.y].x, Lb[kk2.y].y};
                    if (wk) {
                        A = cdf{df_mul(A.x, wa), df_mul(A.y, wa)};
                        B = cdf{df_mul(B.x, wb), df_mul(B.y, wb)};
                    }
                    sp[v * kRC + r] = cdf{df_add(A.x, B.x), df_add(A.y, B.y)};    // P = A + B
                    siq[v * kRC + r] = cdf{df_sub(B.y, A.y), df_sub(A.x, B.x)};   // i Q, Q = A - B
                }
            }
            __syncwarp();
            if (active)
                for (int kk = 0; kk < pn; ++kk) {
                    const cdf e = cis_turns_big(df_dot3(&ss[3 * kk], d), tab);
                    for (int r = 0; r < rn; ++r) {
                        const cdf P = sp[kk * kRC + r], iQ = siq[kk * kRC + r];
                        dfacc_add_prod(ax[r], P.x, e.x);
                        dfacc_add_prod(ax[r], iQ.x, e.y);
                        dfacc_add_prod(ay[r], P.y, e.x);
                        dfacc_add_prod(ay[r], iQ.y, e.y);
                    }
                }
        }
        if (active)
            for (int r = 0; r < rn; ++r) {
                cxd& o = out[(int64_t)(t0 + ti) * R_ + r0 + r];
                o.x += df_to_double(dfacc_get(ax[r]));
                o.y += df_to_double(dfacc_get(ay[r]));
            }
    }
}

// mixed near field, one warp per (target box, 32-target chunk); float32 sums over tiles of
// kWarpTile sources, flushed into float64
template <int kRC>   // right-hand sides per pass: 1 (single RHS) or 4
__global__ void __launch_bounds__(128) k_p2p_mixed_warp(
    const int2* __restrict__ units, int nunits, const int32_t* __restrict__ tstart,
    const int32_t* __restrict__ tcount, const int32_t* __restrict__ sstart, const int32_t* __restrict__ scount,
    const int32_t* __restrict__ noff, const int32_t* __restrict__ nidx, P2PMixedArgs a,
    const cxd* __restrict__ qs, cxd* __restrict__ phis, int R) {
    __shared__ float4 shp[4][kWarpTile], sho[4][kWarpTile];
    __shared__ cxf shq[4][kWarpTile * kRC];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int u = blockIdx.x * 4 + warp;
    if (u >= nunits) return;
    const int b = units[u].x, c0 = units[u].y;
    const int t0 = tstart[b], tc = tcount[b];
    const int ti = c0 + lane;
    const bool active = ti < tc;
    const float two_pi = 6.28318530717958647692f;
    float4 gp = make_float4(0, 0, 0, 0), op = gp;
    if (active) {
        gp = a.tpt[t0 + ti];
        op = a.tof[t0 + ti];
    }
    float4* wp = shp[warp];
    float4* wo = sho[warp];
    cxf* wq = shq[warp];
    for (int r0 = 0; r0 < R; r0 += kRC) {
        const int rn = kRC == 1 ? 1 : min(kRC, R - r0);
        dfacc ax[kRC], ay[kRC];   // float32 tile sums gathered in double-float
        for (int r = 0; r < kRC; ++r) ax[r] = ay[r] = dfacc{0.f, 0.f};
        for (int nb = noff[b]; nb < noff[b + 1]; ++nb) {
            const int s = nidx[nb];
            const int s0 = sstart[s], sc = scount[s];
            for (int sb = 0; sb < sc; sb += kWarpTile) {
                const int sn = min(kWarpTile, sc - sb);
                __syncwarp();
                for (int v = lane; v < sn; v += 32) {
                    const int j = s0 + sb + v;
                    wp[v] = a.spt[j];
                    wo[v] = a.sof[j];
                    for (int r = 0; r < rn; ++r) wq[v * kRC + r] = cvt<float>(qs[(int64_t)j * R + r0 + r]);
                }
                __syncwarp();
                if (!active) continue;
                cxf tile[kRC];
                for (int r = 0; r < kRC; ++r) tile[r] = mk<float>(0, 0);
                for (int jj = 0; jj < sn; ++jj) {
                    const float4 sp = wp[jj], so = wo[jj];
                    const float Dx = gp.x - sp.x, Dy = gp.y - sp.y, Dz = gp.z - sp.z;  // exact
                    const float ex = op.x - so.x, ey = op.y - so.y, ez = op.z - so.z;
                    const float A = fmaf(Dx, Dx, fmaf(Dy, Dy, Dz * Dz));           // exact
                    const float B = fmaf(ex, fmaf(2.0f, Dx, ex),
                                         fmaf(ey, fmaf(2.0f, Dy, ey), ez * fmaf(2.0f, Dz, ez)));
                    const float s2 = A + B;
                    if (s2 <= 0.0f) continue;
                    const float rho = rsqrt_hw(s2);
                    const float r0f = s2 * rho;
                    const float e = fmaf(-r0f, r0f, A);
                    const float c = (e + B) * (0.5f * rho);
                    const float th = a.tau_hi * r0f;
                    float te = fmaf(a.tau_hi, r0f, -th);
                    te = fmaf(a.tau_hi, c, te);
                    te = fmaf(a.tau_lo, r0f, te);
                    const float f = (th - rintf(th)) + te;
                    float sn_, cs_;
                    sincos_hw(two_pi * f, &sn_, &cs_);
                    const cxf g = mk<float>(cs_ * rho, sn_ * rho);
                    if (kRC == 1) mac(tile[0], g, wq[jj]);
                    else
                        for (int r = 0; r < rn; ++r) mac(tile[r], g, wq[jj * kRC + r]);
                }
                for (int r = 0; r < rn; ++r) {
                    dfacc_add(ax[r], df{tile[r].x, 0.f});
                    dfacc_add(ay[r], df{tile[r].y, 0.f});
                }
            }
        }
        if (active)
            for (int r = 0; r < rn; ++r)
                phis[(int64_t)(t0 + ti) * R + r0 + r] =
                    mk<double>(a.inv_unit * df_to_double(dfacc_get(ax[r])), a.inv_unit * df_to_double(dfacc_get(ay[r])));
    }
}

// ---------------------------------------------------------------------------
// Symmetric mixed near field (sources = targets, one right-hand side).  G is symmetric,
// so the units of box b evaluate each pair with a neighbour s > b once and use it both
// ways: phi_i += G_ij q_j in registers, phi_j += G_ij q_i summed over the warp's 32
// targets for groups of 8 sources (recursive halving with shuffles, then a butterfly)
// and added atomically; pairs inside box b run one way.  phi must be zero on entry.
// ---------------------------------------------------------------------------
__device__ __forceinline__ cxf sel(bool c, cxf a, cxf b) { return c ? a : b; }

// sum of v[k] over the warp for k = 0..7; lane l returns the total of k = (l >> 2) & 7
__device__ __forceinline__ cxf warp_reduce8(cxf v[8], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const cxf send = sel(b4, v[i], v[i + 4]), keep = sel(b4, v[i + 4], v[i]);
        v[i] = mk<float>(keep.x + __shfl_xor_sync(0xffffffffu, send.x, 16),
                         keep.y + __shfl_xor_sync(0xffffffffu, send.y, 16));
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const cxf send = sel(b3, v[i], v[i + 2]), keep = sel(b3, v[i + 2], v[i]);
        v[i] = mk<float>(keep.x + __shfl_xor_sync(0xffffffffu, send.x, 8),
                         keep.y + __shfl_xor_sync(0xffffffffu, send.y, 8));
    }
    const cxf send = sel(b2, v[0], v[1]), keep = sel(b2, v[1], v[0]);
    cxf r = mk<float>(keep.x + __shfl_xor_sync(0xffffffffu, send.x, 4),
                      keep.y + __shfl_xor_sync(0xffffffffu, send.y, 4));
    r.x += __shfl_xor_sync(0xffffffffu, r.x, 2);
    r.y += __shfl_xor_sync(0xffffffffu, r.y, 2);
    r.x += __shfl_xor_sync(0xffffffffu, r.x, 1);
    r.y += __shfl_xor_sync(0xffffffffu, r.y, 1);
    return r;
}

// float32 kernel value of the exact-grid form (target grid/offset gp, op; source sp, so);
// zero for coincident points
__device__ __forceinline__ cxf green_grid(float4 gp, float4 op, float4 sp, float4 so, float tau_hi,
                                          float tau_lo) {
    const float Dx = gp.x - sp.x, Dy = gp.y - sp.y, Dz = gp.z - sp.z;  // exact
    const float ex = op.x - so.x, ey = op.y - so.y, ez = op.z - so.z;
    const float A = fmaf(Dx, Dx, fmaf(Dy, Dy, Dz * Dz));           // exact
    const float B = fmaf(ex, fmaf(2.0f, Dx, ex), fmaf(ey, fmaf(2.0f, Dy, ey), ez * fmaf(2.0f, Dz, ez)));
    const float s2 = A + B;
    const float rho = s2 > 0.0f ? rsqrt_hw(s2) : 0.0f;
    const float r0f = s2 * rho;
    const float e = fmaf(-r0f, r0f, A);
    const float c = (e + B) * (0.5f * rho);
    const float th = tau_hi * r0f;
    float te = fmaf(tau_hi, r0f, -th);
    te = fmaf(tau_hi, c, te);
    te = fmaf(tau_lo, r0f, te);
    const float f = (th - rintf(th)) + te;
    float sn, cs;
    sincos_hw(6.28318530717958647692f * f, &sn, &cs);
    return mk<float>(cs * rho, sn * rho);
}

// one warp per (box, 32-target chunk).  kMinBlocks: resident blocks per SM the register
// allocation is sized for (the plan times the instantiations on its own near field and keeps
// the fastest; the arithmetic is the same in all of them)
template <int kMinBlocks>
__global__ void __launch_bounds__(128, kMinBlocks) k_p2p_mixed_sym_warp(
    const int2* __restrict__ units, int nunits, const int32_t* __restrict__ start,
    const int32_t* __restrict__ count, const int32_t* __restrict__ noff, const int32_t* __restrict__ nidx,
    P2PMixedArgs a, const cxd* __restrict__ qs, cxd* __restrict__ phis) {
    __shared__ float4 shp[4][kWarpTile], sho[4][kWarpTile];
    __shared__ cxf shq[4][kWarpTile];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int u = blockIdx.x * 4 + warp;
    if (u >= nunits) return;                       // warp-uniform
    const int b = units[u].x, c0 = units[u].y;
    const int t0 = start[b], tc = count[b];
    const int ti = c0 + lane;
    const bool active = ti < tc;
    float4 gp = make_float4(0, 0, 0, 0), op = gp;
    cxf qi = mk<float>(0, 0);
    if (active) {
        gp = a.tpt[t0 + ti];
        op = a.tof[t0 + ti];
        qi = cvt<float>(qs[t0 + ti]);
    }
    float4* wp = shp[warp];
    float4* wo = sho[warp];
    cxf* wq = shq[warp];
    dfacc ax = {0.f, 0.f}, ay = {0.f, 0.f};      // float32 tile sums gathered in double-float
    for (int nb = noff[b]; nb < noff[b + 1]; ++nb) {
        const int s = nidx[nb];
        if (s < b) continue;                       // that pair belongs to box s's units
        const bool both = s > b;
        const int s0 = start[s], sc = count[s];
        for (int sb = 0; sb < sc; sb += kWarpTile) {
            const int sn = min(kWarpTile, sc - sb);
            __syncwarp();
            for (int v = lane; v < sn; v += 32) {
                const int j = s0 + sb + v;
                wp[v] = a.spt[j];
                wo[v] = a.sof[j];
                wq[v] = cvt<float>(qs[j]);
            }
            __syncwarp();
            cxf tile = mk<float>(0, 0);
            for (int jg = 0; jg < sn; jg += 8) {
                // inactive lanes have qi = 0 (and a finite g), so their reverse terms vanish
                cxf rv[8];
                if (jg + 8 <= sn) {                // full group: no per-source bound test
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const cxf g = green_grid(gp, op, wp[jg + k], wo[jg + k], a.tau_hi, a.tau_lo);
                        mac(tile, g, wq[jg + k]);
                        rv[k] = g * qi;
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        rv[k] = mk<float>(0, 0);
                        const int jj = jg + k;
                        if (jj < sn) {             // warp-uniform
                            const cxf g = green_grid(gp, op, wp[jj], wo[jj], a.tau_hi, a.tau_lo);
                            mac(tile, g, wq[jj]);
                            rv[k] = g * qi;
                        }
                    }
                }
                if (both) {                        // warp-uniform
                    const cxf r = warp_reduce8(rv, lane);
                    const int k = (lane >> 2) & 7;
                    if ((lane & 3) == 0 && jg + k < sn) {
                        cxd* o = phis + (s0 + sb + jg + k);
                        atomicAdd(&o->x, f2d_bits(a.inv_unit_f * r.x));
                        atomicAdd(&o->y, f2d_bits(a.inv_unit_f * r.y));
                    }
                }
            }
            dfacc_add(ax, df{tile.x, 0.f});
            dfacc_add(ay, df{tile.y, 0.f});
        }
    }
    if (active) {
        atomicAdd(&phis[t0 + ti].x, a.inv_unit * df_to_double(dfacc_get(ax)));
        atomicAdd(&phis[t0 + ti].y, a.inv_unit * df_to_double(dfacc_get(ay)));
    }
}

// ---------------------------------------------------------------------------
// Mixed near field as a tensor-core GEMM form (many right-hand sides): for a tile of 16
// targets and 8 sources the float32 kernel values G (exact-grid form, as above) are the A
// operand of mma.sync m16n8k8 (TF32), the charges Q of 8 right-hand sides the B operand.
// Each real product is split 3xTF32 (hi*hi + hi*lo + lo*hi, float32 accumulation), so the
// GEMM keeps float32 accuracy; the complex product takes four real ones (Gr Qr - Gi Qi,
// Gr Qi + Gi Qr).  One block per (target box, 64 targets): 4 warps x 16 targets, sources
// staged by the block 32 at a time; float32 sums of each 32-source tile are gathered in
// double-float accumulators in shared memory (per lane, [element][lane] layout).
// Fragment layouts (PTX ISA, mma.m16n8k8 .tf32): g = lane / 4, c = lane % 4;
// A: a0 (g, c), a1 (g+8, c), a2 (g, c+4), a3 (g+8, c+4); B: b0 (c, g), b1 (c+4, g);
// C: c0 (g, 2c), c1 (g, 2c+1), c2 (g+8, 2c), c3 (g+8, 2c+1).
// ---------------------------------------------------------------------------
constexpr int kTcRhs = 32;              // right-hand sides per pass (4 n-tiles of 8)
constexpr int kTcSrc = 32;              // sources staged per block step
constexpr int kTcQStride = kTcRhs + 8;  // padded row: B-fragment loads hit 32 distinct banks
constexpr int kTcAccPerWarp = 2 * 2 * 4 * (kTcRhs / 8) * 32;   // floats of df accumulators per warp
constexpr size_t kTcDynSmem = 4 * kTcAccPerWarp * sizeof(float);

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
    hi = tf32_rna(x);
    lo = tf32_rna(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(128) k_p2p_mixed_tc(
    const int2* __restrict__ units, int nunits, const int32_t* __restrict__ tstart,
    const int32_t* __restrict__ tcount, const int32_t* __restrict__ sstart, const int32_t* __restrict__ scount,
    const int32_t* __restrict__ noff, const int32_t* __restrict__ nidx, P2PMixedArgs a,
    const cxd* __restrict__ qs, cxd* __restrict__ phis, int R) {
    __shared__ float4 shp[kTcSrc], sho[kTcSrc];
    __shared__ float shq[4][kTcSrc * kTcQStride];   // Qr hi, Qr lo, Qi hi, Qi lo (tf32 bits)
    extern __shared__ float acc_dyn[];              // [warp][element][lane]: df (hi, lo) of C
    const int u = blockIdx.x;
    if (u >= nunits) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, c = lane & 3;
    const int b = units[u].x, c0 = units[u].y + 16 * warp;
    const int t0 = tstart[b], tc = tcount[b];
    // this lane's two target rows g and g + 8
    float4 gp[2], op[2];
    bool act[2];
    for (int h = 0; h < 2; ++h) {
        const int ti = c0 + g + 8 * h;
        act[h] = ti < tc;
        gp[h] = op[h] = make_float4(0, 0, 0, 0);
        if (act[h]) {
            gp[h] = a.tpt[t0 + ti];
            op[h] = a.tof[t0 + ti];
        }
    }
    constexpr int kNT = kTcRhs / 8;
    float* ac = acc_dyn + (size_t)warp * kTcAccPerWarp;
    for (int r0 = 0; r0 < R; r0 += kTcRhs) {
        for (int e = 0; e < 2 * 2 * 4 * kNT; ++e) ac[e * 32 + lane] = 0.f;
        for (int nb = noff[b]; nb < noff[b + 1]; ++nb) {
            const int s = nidx[nb];
            const int s0 = sstart[s], sc = scount[s];
            for (int sb = 0; sb < sc; sb += kTcSrc) {
                const int sn = min(kTcSrc, sc - sb);
                __syncthreads();
                for (int v = threadIdx.x; v < kTcSrc; v += blockDim.x) {
                    shp[v] = v < sn ? a.spt[s0 + sb + v] : make_float4(0, 0, 0, 0);
                    sho[v] = v < sn ? a.sof[s0 + sb + v] : make_float4(0, 0, 0, 0);
                }
                for (int v = threadIdx.x; v < kTcSrc * kTcRhs; v += blockDim.x) {
                    const int j = v / kTcRhs, r = v % kTcRhs;
                    float qx = 0.f, qy = 0.f;
                    if (j < sn && r0 + r < R) {
                        const cxd qq = qs[(int64_t)(s0 + sb + j) * R + r0 + r];
                        qx = (float)qq.x;
                        qy = (float)qq.y;
                    }
                    uint32_t h0, l0, h1, l1;
                    tf32_split(qx, h0, l0);
                    tf32_split(qy, h1, l1);
                    shq[0][j * kTcQStride + r] = __uint_as_float(h0);
                    shq[1][j * kTcQStride + r] = __uint_as_float(l0);
                    shq[2][j * kTcQStride + r] = __uint_as_float(h1);
                    shq[3][j * kTcQStride + r] = __uint_as_float(l1);
                }
                __syncthreads();
                float cr[kNT][4], ci[kNT][4];
                for (int nt = 0; nt < kNT; ++nt)
                    for (int i = 0; i < 4; ++i) cr[nt][i] = ci[nt][i] = 0.f;
                for (int kb = 0; kb < kTcSrc; kb += 8) {
                    if (kb >= sn) break;                       // block-uniform
                    // A fragments: G(row g + 8 (i & 1), source kb + c + 4 (i >> 1))
                    uint32_t grh[4], grl[4], gih[4], gil[4], ngih[4], ngil[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int h = i & 1, jj = kb + c + 4 * (i >> 1);
                        cxf gv = green_grid(gp[h], op[h], shp[jj], sho[jj], a.tau_hi, a.tau_lo);
                        if (!act[h] || jj >= sn) gv = mk<float>(0, 0);
                        tf32_split(gv.x, grh[i], grl[i]);
                        tf32_split(gv.y, gih[i], gil[i]);
                        ngih[i] = gih[i] ^ 0x80000000u;           // -Gi (sign flip is exact)
                        ngil[i] = gil[i] ^ 0x80000000u;
                    }
#pragma unroll
                    for (int nt = 0; nt < kNT; ++nt) {
                        const int col = nt * 8 + g;
                        const int rA = (kb + c) * kTcQStride + col, rB = (kb + c + 4) * kTcQStride + col;
                        const uint32_t qrh0 = __float_as_uint(shq[0][rA]), qrh1 = __float_as_uint(shq[0][rB]);
                        const uint32_t qrl0 = __float_as_uint(shq[1][rA]), qrl1 = __float_as_uint(shq[1][rB]);
                        const uint32_t qih0 = __float_as_uint(shq[2][rA]), qih1 = __float_as_uint(shq[2][rB]);
                        const uint32_t qil0 = __float_as_uint(shq[3][rA]), qil1 = __float_as_uint(shq[3][rB]);
                        // real part: Gr Qr - Gi Qi
                        mma_tf32(cr[nt], grh, qrh0, qrh1);
                        mma_tf32(cr[nt], grh, qrl0, qrl1);
                        mma_tf32(cr[nt], grl, qrh0, qrh1);
                        mma_tf32(cr[nt], ngih, qih0, qih1);
                        mma_tf32(cr[nt], ngih, qil0, qil1);
                        mma_tf32(cr[nt], ngil, qih0, qih1);
                        // imaginary part: Gr Qi + Gi Qr
                        mma_tf32(ci[nt], grh, qih0, qih1);
                        mma_tf32(ci[nt], grh, qil0, qil1);
                        mma_tf32(ci[nt], grl, qih0, qih1);
                        mma_tf32(ci[nt], gih, qrh0, qrh1);
                        mma_tf32(ci[nt], gih, qrl0, qrl1);
                        mma_tf32(ci[nt], gil, qrh0, qrh1);
                    }
                }
                // float32 tile sums into the double-float accumulators (lane-private entries)
#pragma unroll
                for (int nt = 0; nt < kNT; ++nt)
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int e = (nt * 4 + i) * 4;
                        dfacc x = {ac[(e + 0) * 32 + lane], ac[(e + 1) * 32 + lane]};
                        dfacc y = {ac[(e + 2) * 32 + lane], ac[(e + 3) * 32 + lane]};
                        dfacc_add(x, df{cr[nt][i], 0.f});
                        dfacc_add(y, df{ci[nt][i], 0.f});
                        ac[(e + 0) * 32 + lane] = x.hi;
                        ac[(e + 1) * 32 + lane] = x.lo;
                        ac[(e + 2) * 32 + lane] = y.hi;
                        ac[(e + 3) * 32 + lane] = y.lo;
                    }
            }
        }
        // C element (nt, i): row g + 8 (i >> 1), column nt * 8 + 2c + (i & 1)
#pragma unroll
        for (int nt = 0; nt < kNT; ++nt)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int h = i >> 1, r = r0 + nt * 8 + 2 * c + (i & 1);
                if (act[h] && r < R) {
                    const int e = (nt * 4 + i) * 4;
                    const double xr = (double)ac[(e + 0) * 32 + lane] + (double)ac[(e + 1) * 32 + lane];
                    const double yi = (double)ac[(e + 2) * 32 + lane] + (double)ac[(e + 3) * 32 + lane];
                    phis[(int64_t)(t0 + c0 + g + 8 * h) * R + r] = mk<double>(a.inv_unit * xr, a.inv_unit * yi);
                }
            }
    }
}

// ---------------------------------------------------------------------------
// near field in double-float (mixed policy, 1e-11 <= eps < 1e-6): positions as df pairs
// relative to the root corner; one warp per (target box, 32-target chunk).
// ---------------------------------------------------------------------------
// G = exp(i k R) / R for the df difference d; false when R = 0.  R and 1/R: the float
// rsqrt seed y refined by one Newton step each (relative error about 1.5 x the seed's
// squared, below 2^-41 for a seed within 2 ulp).
__device__ __forceinline__ bool green_df(const df* d, df kt, const cdf* tab, cdf& g) {
    const df r2 = df_dot3(d, d);
    if (!(r2.hi > 0.0f)) return false;
    const float y = rsqrtf(r2.hi);
    const float r0 = __fmul_rn(r2.hi, y);
    const float p = __fmul_rn(r0, r0);
    const float pe = __fmaf_rn(r0, r0, -p);
    const float res = __fadd_rn(__fsub_rn(__fsub_rn(r2.hi, p), pe), r2.lo);     // r2 - r0^2
    const df R = df_fast_sum(r0, __fmul_rn(res, __fmul_rn(0.5f, y)));
    const float q = __fmul_rn(R.hi, y);
    const float qe = __fmaf_rn(R.hi, y, -q);
    const float e = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, q), qe), __fmul_rn(R.lo, y));  // 1 - R y
    const df inv = df_fast_sum(y, __fmul_rn(y, e));
    const cdf c = cis_turns_big(df_mul(R, kt), tab);
    g = cdf{df_mul(c.x, inv), df_mul(c.y, inv)};
    return true;
}

template <int kRC>   // right-hand sides per pass: 1 (single RHS) or 4
__global__ void __launch_bounds__(128) k_p2p_df_warp(
    const int2* __restrict__ units, int nunits, const int32_t* __restrict__ tstart,
    const int32_t* __restrict__ tcount, const int32_t* __restrict__ sstart, const int32_t* __restrict__ scount,
    const int32_t* __restrict__ noff, const int32_t* __restrict__ nidx, const df* __restrict__ tpos,
    const df* __restrict__ spos, df kt, const cdf* __restrict__ cis_tab, const cxd* __restrict__ qs,
    cxd* __restrict__ phis, int R) {
    __shared__ cdf tab[kCisTableBig];
    __shared__ df shp[4][kWarpTile * 3];
    __shared__ cdf shq[4][kWarpTile * kRC];
    for (int v = threadIdx.x; v < kCisTableBig; v += blockDim.x) tab[v] = cis_tab[v];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int u = blockIdx.x * 4 + warp;
    if (u >= nunits) return;
    const int b = units[u].x, c0 = units[u].y;
    const int t0 = tstart[b], tc = tcount[b];
    const int ti = c0 + lane;
    const bool active = ti < tc;
    df x[3] = {{0, 0}, {0, 0}, {0, 0}};
    if (active)
        for (int c = 0; c < 3; ++c) x[c] = tpos[3 * (int64_t)(t0 + ti) + c];
    df* wp = shp[warp];
    cdf* wq = shq[warp];
    for (int r0 = 0; r0 < R; r0 += kRC) {
        const int rn = kRC == 1 ? 1 : min(kRC, R - r0);
        cxd acc[kRC];
        for (int r = 0; r < kRC; ++r) acc[r] = mk<double>(0, 0);
        for (int nb = noff[b]; nb < noff[b + 1]; ++nb) {
            const int s = nidx[nb];
            const int s0 = sstart[s], sc = scount[s];
            for (int sb = 0; sb < sc; sb += kWarpTile) {
                const int sn = min(kWarpTile, sc - sb);
                __syncwarp();
                for (int v = lane; v < sn; v += 32) {
                    const int64_t j = s0 + sb + v;
                    for (int c = 0; c < 3; ++c) wp[3 * v + c] = spos[3 * j + c];
                    for (int r = 0; r < rn; ++r) {
                        const cxd qq = qs[j * R + r0 + r];
                        wq[v * kRC + r] = cdf{df_from_double(qq.x), df_from_double(qq.y)};
                    }
                }
                __syncwarp();
                if (!active) continue;
                dfacc ax[kRC], ay[kRC];
                for (int r = 0; r < kRC; ++r) ax[r] = ay[r] = dfacc{0.f, 0.f};
                for (int jj = 0; jj < sn; ++jj) {
                    const df d[3] = {df_sub(x[0], wp[3 * jj]), df_sub(x[1], wp[3 * jj + 1]),
                                     df_sub(x[2], wp[3 * jj + 2])};
                    cdf g;
                    if (!green_df(d, kt, tab, g)) continue;
                    for (int r = 0; r < rn; ++r) {
                        const cdf q = wq[jj * kRC + r];
                        dfacc_add_prod(ax[r], g.x, q.x);
                        dfacc_add_prod(ax[r], df_neg(g.y), q.y);
                        dfacc_add_prod(ay[r], g.x, q.y);
                        dfacc_add_prod(ay[r], g.y, q.x);
                    }
                }
                for (int r = 0; r < rn; ++r) {
                    acc[r].x += df_to_double(dfacc_get(ax[r]));
                    acc[r].y += df_to_double(dfacc_get(ay[r]));
                }
            }
        }
        if (active)
            for (int r = 0; r < rn; ++r) phis[(int64_t)(t0 + ti) * R + r0 + r] = acc[r];
    }
}

// ---------------------------------------------------------------------------
// Position gradient (vector-Jacobian product of phi = A(y) q for a real loss, with
// g = dL/d conj(phi) in the convention of complex autograd):
//   grad_j = Re[ sum_r q_jr ( i k sum_k s_k exp(i k s_k.(y_j - c_b)) Lambda_b,r(k)
//                             + sum_{i in N(b)} conj(g_ir) dG(x_i, y_j)/dy_j ) ]
// with Lambda = the transposed far-field chain applied to conj(g) and
// dG/dy = G (i k - 1/R) (y - x) / R.
// ---------------------------------------------------------------------------
template <typename S, typename R>
__global__ void k_grad_far(BoxView bx, QuadView qv, const int32_t* __restrict__ sstart,
                           const int32_t* __restrict__ scount, const double* __restrict__ sx,
                           const double* __restrict__ sy, const double* __restrict__ sz,
                           const cx<S>* __restrict__ Lam, const cxd* __restrict__ qs, int R_, double kappa,
                           double* __restrict__ grad) {
    __shared__ double shs[kL2TThreads * 3];
    __shared__ cx<R> shl[kL2TThreads];
    const int b = bx.leaf ? bx.leaf[blockIdx.x] : (int)blockIdx.x;
    const int s0 = sstart[b], sc = scount[b];
    if ((int)blockIdx.y * kL2TThreads >= sc) return;
    const double kt = kappa / (2.0 * 3.14159265358979323846);
    const double cxx = bx.center[3 * b], cyy = bx.center[3 * b + 1], czz = bx.center[3 * b + 2];
    {
        const int jb = blockIdx.y * kL2TThreads;
        const int jj = jb + threadIdx.x;
        const bool active = jj < sc;
        double d[3] = {0, 0, 0};
        if (active) {
            d[0] = sx[s0 + jj] - cxx;
            d[1] = sy[s0 + jj] - cyy;
            d[2] = sz[s0 + jj] - czz;
        }
        double g[3] = {0, 0, 0};
        for (int r = 0; r < R_; ++r) {
            const cx<S>* Lb = Lam + ((int64_t)b * R_ + r) * qv.K;
            cxd acc[3] = {mk<double>(0, 0), mk<double>(0, 0), mk<double>(0, 0)};
            for (int64_t kb = 0; kb < qv.K; kb += kL2TThreads) {
                const int kn = (int)min((int64_t)kL2TThreads, qv.K - kb);
                __syncthreads();
                if (threadIdx.x < kn) {
                    const int64_t k = kb + threadIdx.x;
                    for (int c = 0; c < 3; ++c) shs[3 * threadIdx.x + c] = qv.shat[3 * k + c];
                    shl[threadIdx.x] = cvt<R>(Lb[k]);
                }
                __syncthreads();
                if (active)
                    for (int kk = 0; kk < kn; ++kk) {
                        double t = turns(kt, &shs[3 * kk], d[0], d[1], d[2]);
                        cx<R> e = plane_wave<R>(t) * shl[kk];
                        for (int c = 0; c < 3; ++c) {
                            acc[c].x += shs[3 * kk + c] * (double)e.x;
                            acc[c].y += shs[3 * kk + c] * (double)e.y;
                        }
                    }
            }
            if (active) {
                const cxd q = qs[(int64_t)(s0 + jj) * R_ + r];
                for (int c = 0; c < 3; ++c) {
                    // Re[q * i k acc] = -k (q.x acc.y + q.y acc.x)
                    g[c] += -kappa * (q.x * acc[c].y + q.y * acc[c].x);
                }
            }
        }
        if (active)
            for (int c = 0; c < 3; ++c) grad[(int64_t)(s0 + jj) * 3 + c] += g[c];
    }
}

// near-field part; one CTA per source leaf box, targets of the neighbour boxes staged
__global__ void k_grad_near(int nbox, const int32_t* __restrict__ sstart, const int32_t* __restrict__ scount,
                            const int32_t* __restrict__ tstart, const int32_t* __restrict__ tcount,
                            const int32_t* __restrict__ noff, const int32_t* __restrict__ nidx,
                            const double* __restrict__ sx, const double* __restrict__ sy,
                            const double* __restrict__ sz, const double* __restrict__ tx,
                            const double* __restrict__ ty, const double* __restrict__ tz,
                            const cxd* __restrict__ qs, const cxd* __restrict__ gconj, int R_, double kappa,
                            double* __restrict__ grad) {
    __shared__ double shx[kP2PThreads], shy[kP2PThreads], shz[kP2PThreads];
    __shared__ cxd shg[kP2PThreads];
    const int b = blockIdx.x;
    if (b >= nbox) return;
    const int s0 = sstart[b], sc = scount[b];
    if ((int)blockIdx.y * kP2PThreads >= sc) return;
    {
        const int jb = blockIdx.y * kP2PThreads;
        const int jj = jb + threadIdx.x;
        const bool active = jj < sc;
        double y0 = 0, y1 = 0, y2 = 0;
        if (active) {
            y0 = sx[s0 + jj];
            y1 = sy[s0 + jj];
            y2 = sz[s0 + jj];
        }
        double gsum[3] = {0, 0, 0};
        for (int r = 0; r < R_; ++r) {
            cxd acc[3] = {mk<double>(0, 0), mk<double>(0, 0), mk<double>(0, 0)};
            for (int nb = noff[b]; nb < noff[b + 1]; ++nb) {
                const int t = nidx[nb];
                const int t0 = tstart[t], tc = tcount[t];
                for (int ib = 0; ib < tc; ib += kP2PThreads) {
                    const int in = min(kP2PThreads, tc - ib);
                    __syncthreads();
                    if (threadIdx.x < in) {
                        const int i = t0 + ib + threadIdx.x;
                        shx[threadIdx.x] = tx[i];
                        shy[threadIdx.x] = ty[i];
                        shz[threadIdx.x] = tz[i];
                        shg[threadIdx.x] = gconj[(int64_t)i * R_ + r];
                    }
                    __syncthreads();
                    if (active)
                        for (int ii = 0; ii < in; ++ii) {
                            const double dx = y0 - shx[ii], dy = y1 - shy[ii], dz = y2 - shz[ii];
                            const double r2 = dx * dx + dy * dy + dz * dz;
                            if (r2 == 0.0) continue;
                            const double rr = sqrt(r2), inv = 1.0 / rr;
                            double sn_, cs_;
                            sincos(kappa * rr, &sn_, &cs_);
                            // G (i k - 1/R) / R
                            const cxd gk = mk<double>(cs_ * inv, sn_ * inv) * mk<double>(-inv * inv, kappa * inv);
                            const cxd v = gk * shg[ii];
                            acc[0].x += v.x * dx; acc[0].y += v.y * dx;
                            acc[1].x += v.x * dy; acc[1].y += v.y * dy;
                            acc[2].x += v.x * dz; acc[2].y += v.y * dz;
                        }
                }
            }
            if (active) {
                const cxd q = qs[(int64_t)(s0 + jj) * R_ + r];
                for (int c = 0; c < 3; ++c) gsum[c] += q.x * acc[c].x - q.y * acc[c].y;
            }
        }
        if (active)
            for (int c = 0; c < 3; ++c) grad[(int64_t)(s0 + jj) * 3 + c] = gsum[c];
    }
}

__global__ void k_scatter_grad(const double* __restrict__ gs, int64_t n, const int64_t* __restrict__ perm,
                               double* __restrict__ grad) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * 3) return;
    int64_t p = t / 3;
    grad[perm[p] * 3 + (t - p * 3)] = gs[t];
}

// ---------------------------------------------------------------------------
// M2L: I_a(s_k) = sum_{b in I(a)} T^{s,LL}_{v(a,b)}(s_k) M_b(s_k); thread per (box, k)
// ---------------------------------------------------------------------------
// S: storage type of tables and signatures, C: compute type (double-float for float64
// levels of the mixed policy)
// complex multiply-accumulate of the list sum: plain for float / double; for double-float
// the four Dekker products go straight into lazy accumulators (no per-term renormalisation)
template <typename C>
struct M2LAcc {
    cx<C> v;
    __device__ __forceinline__ void zero() { v = mk<C>(rval<C>(0.0), rval<C>(0.0)); }
    __device__ __forceinline__ void mac(cx<C> t, cx<C> m) {   // four FMA
        v.x = fma(t.x, m.x, fma(-t.y, m.y, v.x));
        v.y = fma(t.x, m.y, fma(t.y, m.x, v.y));
    }
    __device__ __forceinline__ cx<C> get() const { return v; }
};
template <>
struct M2LAcc<df> {
    dfacc x, y;
    __device__ __forceinline__ void zero() { x = y = dfacc{0.f, 0.f}; }
    __device__ __forceinline__ void mac(cx<df> t, cx<df> m) {
        dfacc_add_prod(x, t.x, m.x);
        dfacc_add_prod(x, df_neg(t.y), m.y);
        dfacc_add_prod(y, t.x, m.y);
        dfacc_add_prod(y, t.y, m.x);
    }
    __device__ __forceinline__ cx<df> get() const { return mk<df>(dfacc_get(x), dfacc_get(y)); }
};

// M2L per box: one thread per (box, sample) sums its interaction list in list order
// (Morton order); islot is the table slot of every list entry.
template <typename S, typename C, int kRC>
__global__ void k_m2l_box(int64_t K, const int32_t* __restrict__ ioff, const int32_t* __restrict__ iidx,
                          const int32_t* __restrict__ islot, const cx<S>* __restrict__ T,
                          const cx<S>* __restrict__ M, int R_, cx<S>* __restrict__ I) {
    // the box's list passes through shared memory in chunks (one broadcast read per entry
    // instead of two global loads), so the signature loads of several entries can be in flight
    constexpr int kChunk = 256;
    __shared__ int2 sl[kChunk];   // (partner box, table slot)
    const int a = blockIdx.x;
    const int64_t k = blockIdx.y * (int64_t)blockDim.x + threadIdx.x;
    const bool active = k < K;
    const int l0 = ioff[a], l1 = ioff[a + 1];
    for (int r0 = 0; r0 < R_; r0 += kRC) {
        const int rn = min(kRC, R_ - r0);
        M2LAcc<C> acc[kRC];
#pragma unroll
        for (int r = 0; r < kRC; ++r) acc[r].zero();
        for (int t0 = l0; t0 < l1; t0 += kChunk) {
            const int tn = min(kChunk, l1 - t0);
            __syncthreads();
            for (int e = threadIdx.x; e < tn; e += blockDim.x) sl[e] = make_int2(iidx[t0 + e], islot[t0 + e]);
            __syncthreads();
            if (active) {
#pragma unroll 4
                for (int e = 0; e < tn; ++e) {
                    const int2 bs = sl[e];
                    const cx<C> tv = cvt<C>(T[(int64_t)bs.y * K + k]);
#pragma unroll
                    for (int r = 0; r < kRC; ++r)
                        if (r < rn) acc[r].mac(tv, cvt<C>(M[((int64_t)bs.x * R_ + r0 + r) * K + k]));
                }
            }
        }
        if (active)
#pragma unroll
            for (int r = 0; r < kRC; ++r)
                if (r < rn) I[((int64_t)a * R_ + r0 + r) * K + k] = cvt<S>(acc[r].get());
    }
}

// M2L by sibling groups: one block per (parent box, tile of samples) evaluates the lists of
// all children of the parent together.  The children's lists are subsets of one union (the
// children of the parent's neighbours), so each partner signature is read once for all
// siblings that list it (a per-entry mask) instead of once per sibling: with two buffer
// boxes (lists up to 875 entries) the partner reads drop about sevenfold.  Each child still
// sums its own entries in Morton order (the order of its list), as k_m2l_box does, so the two
// give the same result; the plan times both on each level and keeps the faster.
// Union entry e of parent p: box pu[e], children mask pmask[e] (bit c = child c lists it),
// table slot pslot[8 e + c] of child c's transfer vector.
template <typename S, typename C, int kRC>
__global__ void k_m2l_sib(int64_t K, const int32_t* __restrict__ pfirst, const int32_t* __restrict__ pnch,
                          const int32_t* __restrict__ poff, const int32_t* __restrict__ pu,
                          const int32_t* __restrict__ pmask, const int32_t* __restrict__ pslot,
                          const cx<S>* __restrict__ T, const cx<S>* __restrict__ M, int R_,
                          cx<S>* __restrict__ I) {
    // the union entries pass through shared memory in chunks (broadcast reads)
    constexpr int kChunk = 64;
    __shared__ int su[kChunk], smask[kChunk], sslot[8 * kChunk];
    const int p = blockIdx.x;
    const int64_t k = blockIdx.y * (int64_t)blockDim.x + threadIdx.x;
    const bool active = k < K;
    const int c0 = pfirst[p], nc = pnch[p];
    const int e0 = poff[p], e1 = poff[p + 1];
    for (int r0 = 0; r0 < R_; r0 += kRC) {
        const int rn = min(kRC, R_ - r0);
        M2LAcc<C> acc[8][kRC];
#pragma unroll
        for (int c = 0; c < 8; ++c)
#pragma unroll
            for (int r = 0; r < kRC; ++r) acc[c][r].zero();
        for (int q0 = e0; q0 < e1; q0 += kChunk) {
            const int qn = min(kChunk, e1 - q0);
            __syncthreads();
            for (int x = threadIdx.x; x < 8 * qn; x += blockDim.x) sslot[x] = pslot[8 * q0 + x];
            for (int x = threadIdx.x; x < qn; x += blockDim.x) {
                su[x] = pu[q0 + x];
                smask[x] = pmask[q0 + x];
            }
            __syncthreads();
            if (!active) continue;
            for (int e = 0; e < qn; ++e) {
                const int u = su[e], mask = smask[e];
                cx<C> m[kRC];
#pragma unroll
                for (int r = 0; r < kRC; ++r)
                    m[r] = r < rn ? cvt<C>(M[((int64_t)u * R_ + r0 + r) * K + k]) : mk<C>(rval<C>(0.0), rval<C>(0.0));
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    if (mask & (1 << c)) {                 // uniform across the block
                        const cx<C> t = cvt<C>(T[(int64_t)sslot[8 * e + c] * K + k]);
#pragma unroll
                        for (int r = 0; r < kRC; ++r) acc[c][r].mac(t, m[r]);
                    }
            }
        }
        if (!active) continue;
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if (c < nc)
#pragma unroll
                for (int r = 0; r < kRC; ++r)
                    if (r < rn) I[((int64_t)(c0 + c) * R_ + r0 + r) * K + k] = cvt<S>(acc[c][r].get());
    }
}

// ---------------------------------------------------------------------------
// Re-quadrature (Section 3.4) in three passes through global scratch (kernels below):
//   A': rows n of quadrature a, N_phi^a(n) -> band-limited phi coefficients (step 1;
//       optional shift pre-multiply)
//   B': theta circles of coefficient pairs, ntheta^a -> ntheta^b        (steps 2-4)
//   C': rows n' of quadrature b from their coefficients                 (step 5; M2M: shift +
//       child sum, L2L: add the incoming I)
// GA layout: [(seq_box * R + r) * rows_a + n] * big ; GB: [(seq_box * R + r) * rows_b + n] * big
// ---------------------------------------------------------------------------
struct RequadArgs {
    QuadView qa, qb;
    int big;
    int maxlen;       // shared buffer length per warp
    TwiddleView tw;
};

// Shift modes of the passes that touch the parent grid.
enum ShiftMode { kNoShift = 0, kShiftConj = 1, kShiftPlain = 2 };

// ---------------------------------------------------------------------------
// Forward re-quadrature on phi-Fourier coefficients.  The phi re-sampling of a row and the
// theta re-sampling of a column act on different axes, so the theta passes may run on the
// band-limited phi coefficients: the big-grid interpolation of step 1 and the big-length
// transform of step 5 drop out.  Coefficient f sits in slot (f + big) % big; a shift of phi
// by pi multiplies it by (-1)^f, so the theta circle of coefficient f is even (f even) or
// odd (f odd) in theta.  Slots c and big - 1 - c (f = c and f = -(c + 1), opposite parity)
// share one complex circle; the even and odd parts separate after the re-sampling.  Same
// bands as the sample passes: min(ceil(n/2), ceil(n'/2)) - 1 for each 1-D step.
// ---------------------------------------------------------------------------
// Pass A': rows of grid a -> band-limited coefficients (scaled by 1/N_phi) in GA
template <typename Tin, typename Tc, int kShift>
__global__ void k_requad_spec_a(RequadArgs ra, int nbox_seq, int R_, const cx<Tin>* __restrict__ in,
                                const int32_t* __restrict__ src_box, const int32_t* __restrict__ octant,
                                const cx<Tc>* __restrict__ shift, cx<Tc>* __restrict__ GA) {
    extern __shared__ unsigned char smem_raw[];
    cx<Tc>* sm = reinterpret_cast<cx<Tc>*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    cx<Tc>* buf0 = sm + (size_t)warp * 2 * ra.maxlen;
    cx<Tc>* buf1 = buf0 + ra.maxlen;
    const int64_t seq = (int64_t)blockIdx.x * kWarps + warp;
    const int rows = ra.qa.nrows;
    if (seq >= (int64_t)nbox_seq * R_ * rows) return;
    const int n = (int)(seq % rows);
    const int64_t br = seq / rows;
    const int b = (int)(br / R_), r = (int)(br % R_);
    const int len = ra.qa.nphi[n];
    const int64_t o = ra.qa.off[n];
    const int sb = kShift ? src_box[b] : b;
    const cx<Tin>* src = in + ((int64_t)sb * R_ + r) * ra.qa.K + o;
    const cx<Tc>* sh = kShift ? shift + (int64_t)octant[b] * ra.qa.K + o : nullptr;
    for (int j = lane; j < len; j += 32) {
        cx<Tc> v = cvt<Tc>(src[j]);
        if (kShift == kShiftConj) v = v * conj(sh[j]);
        if (kShift == kShiftPlain) v = v * sh[j];
        buf0[j] = v;
    }
    __syncwarp();
    const cx<Tc>* pool = reinterpret_cast<const cx<Tc>*>(ra.tw.pool);
    const cx<Tc>* sp = warp_fft(buf0, buf1, len, false, pool + ra.tw.off[len], lane);
    const int band = min((len + 1) / 2, (ra.big + 1) / 2) - 1;
    const Tc scale = rratio<Tc>(1, len);
    cx<Tc>* dst = GA + seq * ra.big;
    for (int j = lane; j < ra.big; j += 32) {
        const int f = (2 * j <= ra.big) ? j : j - ra.big;
        cx<Tc> v = mk<Tc>(rval<Tc>(0.0), rval<Tc>(0.0));
        if (f <= band && f >= -band) v = scale * sp[(f + len) % len];
        dst[j] = v;
    }
}

// Pass B': one circle per slot pair (c, big - 1 - c), c < big / 2
template <typename Tc>
__global__ void k_requad_spec_cols(RequadArgs ra, int nbox_seq, int R_, const cx<Tc>* __restrict__ GA,
                                   cx<Tc>* __restrict__ GB) {
    extern __shared__ unsigned char smem_raw[];
    cx<Tc>* sm = reinterpret_cast<cx<Tc>*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    cx<Tc>* buf0 = sm + (size_t)warp * 2 * ra.maxlen;
    cx<Tc>* buf1 = buf0 + ra.maxlen;
    const int hb = ra.big / 2;
    const int64_t seq = (int64_t)blockIdx.x * kWarps + warp;
    if (seq >= (int64_t)nbox_seq * R_ * hb) return;
    const int c = (int)(seq % hb);
    const int64_t br = seq / hb;
    // slot c holds f = c, slot big - 1 - c holds f = -(c + 1): opposite parity
    const int s_even = (c % 2 == 0) ? c : ra.big - 1 - c;
    const int s_odd = (c % 2 == 0) ? ra.big - 1 - c : c;
    const int nta = ra.qa.ntheta, ntb = ra.qb.ntheta;
    const int ha = nta / 2, hbr = ntb / 2;
    const cx<Tc>* ga = GA + br * (int64_t)ra.qa.nrows * ra.big;
    for (int t = lane; t < nta; t += 32) {
        const int u = (t <= ha) ? t : nta - t;
        const cx<Tc> e = ga[(int64_t)u * ra.big + s_even], d = ga[(int64_t)u * ra.big + s_odd];
        buf0[t] = (t <= ha) ? e + d : e - d;    // the odd circle changes sign past theta = pi
    }
    __syncwarp();
    cx<Tc>* res = warp_resample(buf0, buf1, nta, ntb, ra.tw, lane);
    const Tc half = rval<Tc>(0.5);
    cx<Tc>* gb = GB + br * (int64_t)ra.qb.nrows * ra.big;
    for (int n = lane; n <= hbr; n += 32) {
        const cx<Tc> y = res[n], ym = res[(ntb - n) % ntb];
        gb[(int64_t)n * ra.big + s_even] = half * (y + ym);
        gb[(int64_t)n * ra.big + s_odd] = half * (y - ym);
    }
}

// Pass B' of float32 re-quadratures with short theta circles (both N_theta <= 64): the map
// k_requad_spec_cols applies to a coefficient pair (slot se of even, so of odd parity) is
// linear in the pair's two columns of GA, so it is applied as a dense product with 2 x 2 blocks
// of real matrices, W[n][u] = (Lee, Leo, Loe, Loo), built at plan time in float64 by running
// that pass on unit columns:
//     GB[n][se] = sum_u Lee[n][u] GA[u][se] + Leo[n][u] GA[u][so],
//     GB[n][so] = sum_u Loe[n][u] GA[u][se] + Loo[n][u] GA[u][so],   n <= N_theta^b / 2.
// For circles this short a warp-wide FFT leaves most lanes idle; here one thread takes one
// (box, pair, real or imaginary part).  W sits in shared memory, kNR columns per row (zeros
// past nra).  The transposed pass (k_requad_spec_cols_t, GB -> GA) runs the same kernel with
// its own matrices: `in` has nra rows per (box, RHS), `out` nrb, both big slots wide.
constexpr int kThetaDenseMax = 33;   // rows N_theta / 2 + 1 of either grid
template <int kNR>
__global__ void __launch_bounds__(128) k_requad_theta_dense(RequadArgs ra, int64_t nseq, const float4* __restrict__ W,
                                                            int nra, int nrb, const cxf* __restrict__ GA,
                                                            cxf* __restrict__ GB) {
    // GA: input rows (nra per box-RHS), GB: output rows (nrb)
    extern __shared__ float4 sW[];   // [nrb][kNR]
    for (int i = threadIdx.x; i < nrb * kNR; i += blockDim.x) {
        const int n = i / kNR, u = i % kNR;
        sW[i] = u < nra ? W[n * nra + u] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    const int hb = ra.big / 2;
    const int64_t total = nseq * hb * 2;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < total; w += (int64_t)gridDim.x * blockDim.x) {
        const int part = (int)(w & 1);
        const int64_t cb = w >> 1;
        const int c = (int)(cb % hb);
        const int64_t br = cb / hb;
        const int s_even = (c % 2 == 0) ? c : ra.big - 1 - c;
        const int s_odd = (c % 2 == 0) ? ra.big - 1 - c : c;
        const float* ga = reinterpret_cast<const float*>(GA + br * (int64_t)nra * ra.big) + part;
        float ge[kNR], go[kNR];
#pragma unroll
        for (int u = 0; u < kNR; ++u) {
            ge[u] = u < nra ? ga[2 * ((int64_t)u * ra.big + s_even)] : 0.f;
            go[u] = u < nra ? ga[2 * ((int64_t)u * ra.big + s_odd)] : 0.f;
        }
        float* gb = reinterpret_cast<float*>(GB + br * (int64_t)nrb * ra.big) + part;
        for (int n = 0; n < nrb; ++n) {
            const float4* wr = sW + n * kNR;
            float e = 0.f, o = 0.f;
#pragma unroll
            for (int u = 0; u < kNR; ++u) {
                const float4 m = wr[u];
                e = fmaf(m.x, ge[u], fmaf(m.y, go[u], e));
                o = fmaf(m.z, ge[u], fmaf(m.w, go[u], o));
            }
            gb[2 * ((int64_t)n * ra.big + s_even)] = e;
            gb[2 * ((int64_t)n * ra.big + s_odd)] = o;
        }
    }
}

// coefficients of a GB' row, limited to the band of a length-len output row, into buf (length len)
template <typename Tc>
__device__ __forceinline__ void spec_row_to_buf(const cx<Tc>* row, int big, int len, cx<Tc>* buf, int lane) {
    const int band = min((big + 1) / 2, (len + 1) / 2) - 1;
    for (int j = lane; j < len; j += 32) {
        const int f = (2 * j <= len) ? j : j - len;
        cx<Tc> v = mk<Tc>(rval<Tc>(0.0), rval<Tc>(0.0));
        if (f <= band && f >= -band) v = row[(f + big) % big];
        buf[j] = v;
    }
}

// Pass C' (L2L): L_child = rows of grid b from the coefficients + I_child, in place
template <typename Tc, typename Tout>
__global__ void k_requad_spec_c_l2l(RequadArgs ra, int nbox_seq, int R_, const cx<Tc>* __restrict__ GB,
                                    cx<Tout>* __restrict__ IL) {
    extern __shared__ unsigned char smem_raw[];
    cx<Tc>* sm = reinterpret_cast<cx<Tc>*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    cx<Tc>* buf0 = sm + (size_t)warp * 2 * ra.maxlen;
    cx<Tc>* buf1 = buf0 + ra.maxlen;
    const int rows = ra.qb.nrows;
    const int64_t seq = (int64_t)blockIdx.x * kWarps + warp;
    if (seq >= (int64_t)nbox_seq * R_ * rows) return;
    const int n = (int)(seq % rows);
    const int64_t br = seq / rows;
    const int len = ra.qb.nphi[n];
    spec_row_to_buf(GB + seq * ra.big, ra.big, len, buf0, lane);
    __syncwarp();
    const cx<Tc>* pool = reinterpret_cast<const cx<Tc>*>(ra.tw.pool);
    const cx<Tc>* res = warp_fft(buf0, buf1, len, true, pool + ra.tw.off[len], lane);
    cx<Tout>* dst = IL + br * ra.qb.K + ra.qb.off[n];
    for (int j = lane; j < len; j += 32) dst[j] = dst[j] + cvt<Tout>(res[j]);
}

// Pass C' (M2M): M_parent = sum over children of shift * (rows of grid b from the coefficients)
template <typename Tc, typename Tout>
__global__ void k_requad_spec_c_m2m(RequadArgs ra, int nparent, int R_, const int32_t* __restrict__ child_start,
                                    const int32_t* __restrict__ child_count, const int32_t* __restrict__ octant,
                                    const cx<Tc>* __restrict__ shift, const cx<Tc>* __restrict__ GB,
                                    cx<Tout>* __restrict__ Mp) {
    extern __shared__ unsigned char smem_raw[];
    cx<Tc>* sm = reinterpret_cast<cx<Tc>*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    cx<Tc>* buf0 = sm + (size_t)warp * 3 * ra.maxlen;
    cx<Tc>* buf1 = buf0 + ra.maxlen;
    cx<Tc>* acc = buf1 + ra.maxlen;   // sum over children; entry j belongs to lane j % 32
    const int rows = ra.qb.nrows;
    const int64_t seq = (int64_t)blockIdx.x * kWarps + warp;
    if (seq >= (int64_t)nparent * R_ * rows) return;
    const int n = (int)(seq % rows);
    const int64_t pr = seq / rows;
    const int p = (int)(pr / R_), r = (int)(pr % R_);
    const int len = ra.qb.nphi[n];
    const int64_t o = ra.qb.off[n];
    for (int j = lane; j < len; j += 32) acc[j] = mk<Tc>(rval<Tc>(0.0), rval<Tc>(0.0));
    const cx<Tc>* pool = reinterpret_cast<const cx<Tc>*>(ra.tw.pool);
    const int c0 = child_start[p], cn = child_count[p];
    for (int c = c0; c < c0 + cn; ++c) {
        spec_row_to_buf(GB + (((int64_t)c * R_ + r) * rows + n) * ra.big, ra.big, len, buf0, lane);
        __syncwarp();
        const cx<Tc>* res = warp_fft(buf0, buf1, len, true, pool + ra.tw.off[len], lane);
        const cx<Tc>* sh = shift + (int64_t)octant[c] * ra.qb.K + o;
        for (int j = lane; j < len; j += 32) acc[j] = acc[j] + res[j] * sh[j];
        __syncwarp();
    }
    cx<Tout>* dst = Mp + ((int64_t)p * R_ + r) * ra.qb.K + o;
    for (int j = lane; j < len; j += 32) dst[j] = cvt<Tout>(acc[j]);
}

// ---------------------------------------------------------------------------
// Transposed coefficient-space re-quadrature (adjoint and gradient): the exact transposes of
// the passes above, in reverse order.  C'^T: a grid-b row through the unnormalised inverse
// FFT of its length into band slots; B'^T: the transposed even/odd split, the transposed
// theta re-sampling ((ntheta_b / ntheta_a) times the re-sampling back) and the transposed
// gather (a row collects the circle values at t and -t); A'^T: band slots into a row of its
// own length, forward FFT, 1/N_phi.
// ---------------------------------------------------------------------------
template <typename Tin, typename Tc, int kShift>
__global__ void k_requad_spec_ct(RequadArgs ra, int nbox_seq, int R_, const cx<Tin>* __restrict__ in,
                                 const int32_t* __restrict__ src_box, const int32_t* __restrict__ octant,
                                 const cx<Tc>* __restrict__ shift, cx<Tc>* __restrict__ GB) {
    extern __shared__ unsigned char smem_raw[];
    cx<Tc>* sm = reinterpret_cast<cx<Tc>*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    cx<Tc>* buf0 = sm + (size_t)warp * 2 * ra.maxlen;
    cx<Tc>* buf1 = buf0 + ra.maxlen;
    const int64_t seq = (int64_t)blockIdx.x * kWarps + warp;
    const int rows = ra.qb.nrows;
    if (seq >= (int64_t)nbox_seq * R_ * rows) return;
    const int n = (int)(seq % rows);
    const int64_t br = seq / rows;
    const int b = (int)(br / R_), r = (int)(br % R_);
    const int len = ra.qb.nphi[n];
    const int64_t o = ra.qb.off[n];
    const int sb = kShift ? src_box[b] : b;
    const cx<Tin>* src = in + ((int64_t)sb * R_ + r) * ra.qb.K + o;
    const cx<Tc>* sh = kShift ? shift + (int64_t)octant[b] * ra.qb.K + o : nullptr;
    for (int j = lane; j < len; j += 32) {
        cx<Tc> v = cvt<Tc>(src[j]);
        if (kShift == kShiftPlain) v = v * sh[j];
        buf0[j] = v;
    }
    __syncwarp();
    const cx<Tc>* pool = reinterpret_cast<const cx<Tc>*>(ra.tw.pool);
    const cx<Tc>* res = warp_fft(buf0, buf1, len, true, pool + ra.tw.off[len], lane);
    const int band = min((ra.big + 1) / 2, (len + 1) / 2) - 1;
    cx<Tc>* dst = GB + seq * ra.big;
    for (int j = lane; j < ra.big; j += 32) {
        const int f = (2 * j <= ra.big) ? j : j - ra.big;
        cx<Tc> v = mk<Tc>(rval<Tc>(0.0), rval<Tc>(0.0));
        if (f <= band && f >= -band) v = res[(f + len) % len];
        dst[j] = v;
    }
}

template <typename Tc>
__global__ void k_requad_spec_cols_t(RequadArgs ra, int nbox_seq, int R_, const cx<Tc>* __restrict__ GB,
                                     cx<Tc>* __restrict__ GA) {
    extern __shared__ unsigned char smem_raw[];
    cx<Tc>* sm = reinterpret_cast<cx<Tc>*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    cx<Tc>* buf0 = sm + (size_t)warp * 2 * ra.maxlen;
    cx<Tc>* buf1 = buf0 + ra.maxlen;
    const int hb = ra.big / 2;
    const int64_t seq = (int64_t)blockIdx.x * kWarps + warp;
    if (seq >= (int64_t)nbox_seq * R_ * hb) return;
    const int c = (int)(seq % hb);
    const int64_t br = seq / hb;
    const int s_even = (c % 2 == 0) ? c : ra.big - 1 - c;
    const int s_odd = (c % 2 == 0) ? ra.big - 1 - c : c;
    const int nta = ra.qa.ntheta, ntb = ra.qb.ntheta;
    const int ha = nta / 2, hbr = ntb / 2;
    const Tc half = rval<Tc>(0.5);
    const cx<Tc>* gb = GB + br * (int64_t)ra.qb.nrows * ra.big;
    // transposed even/odd split: rows n <= ntheta_b / 2 of the two slots -> one circle
    for (int m = lane; m < ntb; m += 32) {
        cx<Tc> y;
        if (m == 0 || m == hbr) {
            y = gb[(int64_t)m * ra.big + s_even];
        } else {
            const int n = m < hbr ? m : ntb - m;
            const cx<Tc> e = gb[(int64_t)n * ra.big + s_even], d = gb[(int64_t)n * ra.big + s_odd];
            y = half * (m < hbr ? e + d : e - d);
        }
        buf0[m] = y;
    }
    __syncwarp();
    cx<Tc>* res = warp_resample(buf0, buf1, ntb, nta, ra.tw, lane);
    const Tc sc = rratio<Tc>(ntb, nta);
    cx<Tc>* ga = GA + br * (int64_t)ra.qa.nrows * ra.big;
    // transposed gather: row u collects t = u and t = ntheta_a - u (odd slot with a sign flip)
    for (int u = lane; u <= ha; u += 32) {
        const cx<Tc> h0 = res[u];
        const cx<Tc> hm = (u != 0 && u != ha) ? res[nta - u] : mk<Tc>(rval<Tc>(0.0), rval<Tc>(0.0));
        ga[(int64_t)u * ra.big + s_even] = sc * (h0 + hm);
        ga[(int64_t)u * ra.big + s_odd] = sc * (h0 - hm);
    }
}

// band slots of a GA row into a grid-a row of length len, forward FFT, 1/len
template <typename Tc>
__device__ __forceinline__ const cx<Tc>* spec_at_row(const cx<Tc>* row, int big, int len, cx<Tc>* buf0,
                                                     cx<Tc>* buf1, const RequadArgs& ra, int lane) {
    const int band = min((len + 1) / 2, (big + 1) / 2) - 1;
    for (int j = lane; j < len; j += 32) {
        const int f = (2 * j <= len) ? j : j - len;
        cx<Tc> v = mk<Tc>(rval<Tc>(0.0), rval<Tc>(0.0));
        if (f <= band && f >= -band) v = row[(f + big) % big];
        buf0[j] = v;
    }
    __syncwarp();
    const cx<Tc>* pool = reinterpret_cast<const cx<Tc>*>(ra.tw.pool);
    return warp_fft(buf0, buf1, len, false, pool + ra.tw.off[len], lane);
}

// A'^T of the transposed M2M: add into the child's rows
template <typename Tc, typename Tout>
__global__ void k_requad_spec_at_add(RequadArgs ra, int nbox_seq, int R_, const cx<Tc>* __restrict__ GA,
                                     cx<Tout>* __restrict__ out) {
    extern __shared__ unsigned char smem_raw[];
    cx<Tc>* sm = reinterpret_cast<cx<Tc>*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    cx<Tc>* buf0 = sm + (size_t)warp * 2 * ra.maxlen;
    cx<Tc>* buf1 = buf0 + ra.maxlen;
    const int rows = ra.qa.nrows;
    const int64_t seq = (int64_t)blockIdx.x * kWarps + warp;
    if (seq >= (int64_t)nbox_seq * R_ * rows) return;
    const int t = (int)(seq % rows);
    const int64_t br = seq / rows;
    const int len = ra.qa.nphi[t];
    const cx<Tc>* res = spec_at_row(GA + seq * ra.big, ra.big, len, buf0, buf1, ra, lane);
    const Tc sc = rratio<Tc>(1, len);
    cx<Tout>* dst = out + br * ra.qa.K + ra.qa.off[t];
    for (int j = lane; j < len; j += 32) dst[j] = dst[j] + cvt<Tout>(sc * res[j]);
}

// A'^T of the transposed L2L: parent row = sum over children of conj(shift) * (A'^T of the child)
template <typename Tc, typename Tout>
__global__ void k_requad_spec_at_sum(RequadArgs ra, int nparent, int R_, const int32_t* __restrict__ child_start,
                                     const int32_t* __restrict__ child_count, const int32_t* __restrict__ octant,
                                     const cx<Tc>* __restrict__ shift, const cx<Tc>* __restrict__ GA,
                                     cx<Tout>* __restrict__ Mp) {
    extern __shared__ unsigned char smem_raw[];
    cx<Tc>* sm = reinterpret_cast<cx<Tc>*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    cx<Tc>* buf0 = sm + (size_t)warp * 3 * ra.maxlen;
    cx<Tc>* buf1 = buf0 + ra.maxlen;
    cx<Tc>* acc = buf1 + ra.maxlen;
    const int rows = ra.qa.nrows;
    const int64_t seq = (int64_t)blockIdx.x * kWarps + warp;
    if (seq >= (int64_t)nparent * R_ * rows) return;
    const int t = (int)(seq % rows);
    const int64_t pr = seq / rows;
    const int p = (int)(pr / R_), r = (int)(pr % R_);
    const int len = ra.qa.nphi[t];
    const int64_t o = ra.qa.off[t];
    const Tc sc = rratio<Tc>(1, len);
    for (int j = lane; j < len; j += 32) acc[j] = mk<Tc>(rval<Tc>(0.0), rval<Tc>(0.0));
    const int c0 = child_start[p], cn = child_count[p];
    for (int c = c0; c < c0 + cn; ++c) {
        const cx<Tc>* res = spec_at_row(GA + (((int64_t)c * R_ + r) * rows + t) * ra.big, ra.big, len, buf0, buf1,
                                        ra, lane);
        const cx<Tc>* sh = shift + (int64_t)octant[c] * ra.qa.K + o;
        for (int j = lane; j < len; j += 32) acc[j] = acc[j] + (sc * res[j]) * conj(sh[j]);
        __syncwarp();
    }
    cx<Tout>* dst = Mp + ((int64_t)p * R_ + r) * ra.qa.K + o;
    for (int j = lane; j < len; j += 32) dst[j] = cvt<Tout>(acc[j]);
}

}  // namespace hfmm
