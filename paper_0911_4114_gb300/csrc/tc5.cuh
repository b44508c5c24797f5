// Float32 near field for many right-hand sides on the 5th-generation tensor cores
// (tcgen05.mma kind::tf32, accumulators in tensor memory), one persistent CTA per SM.
//
// The near-field sum phi_t,r = sum_s G(x_t, y_s) q_s,r over a target chunk's neighbour
// sources is, for a chunk of 128 targets, a complex GEMM.  Per tile of 16 sources it is done
// as two real GEMMs over K = 32 (the real and imaginary parts of the charges),
//     Re phi[t][r] = sum_j Re G[t][j] Re q[j][r] + (-Im G[t][j]) Im q[j][r],
//     Im phi[t][r] = sum_j Im G[t][j] Re q[j][r] +   Re G[t][j]  Im q[j][r],
// with B[r] = [Re q_r | Im q_r] (64 right-hand sides x 32) shared by both and the A operand of
// each K step of 8 taken from one of three 128 x 16 blocks [Re G | Im G | -Im G] held side by
// side (128 x 48).  Each factor is split into two TF32 parts and three products (hi hi, hi
// lo, lo hi) accumulate in float32 (3xTF32), which keeps float32 accuracy.
//
// The charges do not depend on the target, so their split operand B of every (source tile,
// 64-RHS pass) is written once per apply into global memory in the shared-memory layout
// (k_t5_bsplit, 16 KB per block) and copied into shared memory by one bulk asynchronous copy
// per tile.  The kernel values A depend on both points and are computed in the CTA.  The
// CTA's warps have fixed roles around a ring of three shared-memory stages and three
// tensor-memory accumulators:
//   * 8 producer warps: for each tile wait until its stage is free, start the B copy (one
//     thread), evaluate the 128 x 16 kernel values of the exact-grid float32 form (two threads
//     per target row, 8 sources each), split them and store A hi / lo in the canonical K-major
//     layout without swizzle (8 x 16-byte core matrices; 128 bytes between core matrices along
//     K, one 8-row group after the other);
//   * 1 MMA thread: when a stage's A and B are in and an accumulator is free, issue the 24
//     MMAs (M = 128, N = 64, K = 8; four K steps, three products, real and imaginary part)
//     into a fresh accumulator and commit to the stage's "free" barrier and the accumulator's
//     "full" barrier;
//   * 8 epilogue warps (two per 32-lane quarter of tensor memory, 32 right-hand sides each):
//     read each tile's sums (tcgen05.ld) into float32 registers and release the accumulator;
//     every 64 tiles the registers are added into a float32 block sum held in the last 128
//     columns of tensor memory, and at the end of a (target chunk, pass) the total is written
//     as float64.
// A fresh accumulator per tile keeps the tensor pipe's float32 accumulation short (12
// products per sum; summed over 512 sources in one accumulator it measured 7e-6 relative).
// Every wait gives up after about one second or when another thread of the CTA gave up: the
// CTA then records HFMM's timeout flag, waits (bounded again) for its own copies and MMAs in
// flight, frees its tensor memory and returns.
#pragma once
#include <stdint.h>

#include "cx.cuh"
#include "df.cuh"

namespace hfmm {

constexpr int kT5M = 128;          // targets per CTA tile (MMA M)
constexpr int kT5Src = 16;         // sources per tile (K = 32: real and imaginary parts)
constexpr int kT5Rhs = 64;         // right-hand sides per pass (MMA N = 128)
constexpr int kT5K = 2 * kT5Src;     // B columns: real parts, then imaginary parts
constexpr int kT5AK = 3 * kT5Src;    // A columns: Re G, Im G, -Im G
constexpr int kT5N = 2 * kT5Rhs;     // accumulator columns: Re phi (64), Im phi (64)
constexpr int kT5Stages = 3;       // shared-memory ring
constexpr int kT5Acc = 3;          // tensor-memory accumulators of 128 columns
constexpr uint32_t kT5SumCol = 384;   // float32 block sums: columns 384..511
constexpr uint32_t kT5Cols = 512;     // tensor-memory columns allocated
constexpr int kT5Flush = 64;       // tiles summed in registers between block-sum updates
constexpr int kT5Prod = 8, kT5Epi = 8;   // producer and epilogue warps (then one MMA warp)
constexpr int kT5Threads = 32 * (kT5Prod + kT5Epi + 1);
constexpr uint32_t kT5Lbo = 128;   // bytes between core matrices along K
constexpr uint32_t kT5SboA = (kT5AK / 4) * 128;   // bytes between 8-row groups of A (1536)
constexpr uint32_t kT5SboB = (kT5K / 4) * 128;    // of B (1024)
constexpr size_t kT5OpA = (size_t)kT5M * kT5AK * 4;     // one part of A (24 KB)
constexpr size_t kT5OpB = (size_t)kT5Rhs * kT5K * 4;    // one part of B (8 KB)
constexpr size_t kT5Blk = 2 * kT5OpB;                   // B hi + lo of one (source tile, pass)
constexpr size_t kT5Stage = 2 * kT5OpA + kT5Blk;        // A hi, A lo, B hi, B lo (64 KB)
constexpr size_t kT5Smem = kT5Stages * kT5Stage + 1024;   // + alignment slack
constexpr unsigned long long kT5WaitNs = 1000000000ull;   // give up a wait after 1 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// shared-memory matrix descriptor: start >> 4 (bits 0-13), leading byte offset >> 4 (16-29),
// stride byte offset >> 4 (32-45), fixed 0b001 (46-48), no swizzle
__device__ __forceinline__ uint64_t t5_desc(uint32_t saddr, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(kT5Lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// instruction descriptor of kind::tf32: D float32 (bits 4-5 = 1), A and B TF32 (bits 7-9,
// 10-12 = 2), both K-major, N >> 3 (bits 17-22), M >> 4 (bits 24-28); N = 64
__host__ __device__ constexpr uint32_t t5_idesc() {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kT5Rhs >> 3) << 17) | ((uint32_t)(kT5M >> 4) << 24);
}

__device__ __forceinline__ void t5_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(t5_idesc()), "r"(accumulate));
}

__device__ __forceinline__ void t5_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar));
}

__device__ __forceinline__ bool t5_try_wait(uint32_t mbar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(phase));
    return ok != 0;
}

// bounded wait for the mbarrier phase; false after about kT5WaitNs
__device__ __forceinline__ bool t5_wait(uint32_t mbar, uint32_t phase) {
    const unsigned long long t0 = global_ns();
    while (!t5_try_wait(mbar, phase))
        if (global_ns() - t0 > kT5WaitNs) return false;
    return true;
}

// bounded wait that also gives up when another thread of the CTA has (*abort set); a wait
// that runs out of time sets *abort
__device__ __forceinline__ bool t5_wait_ab(uint32_t mbar, uint32_t phase, volatile int* abort) {
    const unsigned long long t0 = global_ns();
    while (!t5_try_wait(mbar, phase)) {
        if (*abort) return false;
        if (global_ns() - t0 > kT5WaitNs) {
            *abort = 1;
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void t5_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ uint32_t t5_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// byte offset of chunk (row, 4 consecutive K values) in a K-major operand (no swizzle) whose
// 8-row groups are sbo bytes apart
__host__ __device__ __forceinline__ uint32_t t5_off(int row, int chunk, uint32_t sbo) {
    return (uint32_t)(row >> 3) * sbo + (uint32_t)chunk * kT5Lbo + (uint32_t)(row & 7) * 16u;
}

// four values as TF32 hi and lo parts at chunk offset `off` of the hi and lo operands
__device__ __forceinline__ void t5_store4(unsigned char* hi, unsigned char* lo, uint32_t off, float a, float b,
                                          float c, float d) {
    const uint32_t ha = t5_tf32(a), hb = t5_tf32(b), hc = t5_tf32(c), hd = t5_tf32(d);
    uint4 h = make_uint4(ha, hb, hc, hd);
    uint4 l = make_uint4(t5_tf32(a - __uint_as_float(ha)), t5_tf32(b - __uint_as_float(hb)),
                         t5_tf32(c - __uint_as_float(hc)), t5_tf32(d - __uint_as_float(hd)));
    *reinterpret_cast<uint4*>(hi + off) = h;
    *reinterpret_cast<uint4*>(lo + off) = l;
}

// the same four values negated (the TF32 parts of -x are those of x negated)
__device__ __forceinline__ void t5_store4_pair(unsigned char* hi, unsigned char* lo, uint32_t off, uint32_t offneg,
                                               const float* v) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        h[i] = t5_tf32(v[i]);
        l[i] = t5_tf32(v[i] - __uint_as_float(h[i]));
    }
    *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
    const uint32_t sg = 0x80000000u;
    *reinterpret_cast<uint4*>(hi + offneg) = make_uint4(h[0] ^ sg, h[1] ^ sg, h[2] ^ sg, h[3] ^ sg);
    *reinterpret_cast<uint4*>(lo + offneg) = make_uint4(l[0] ^ sg, l[1] ^ sg, l[2] ^ sg, l[3] ^ sg);
}

// float32 kernel value of the exact-grid form (as green_grid in kernels.cuh)
__device__ __forceinline__ cxf t5_green(float4 gp, float4 op, float4 sp, float4 so, float tau_hi, float tau_lo) {
    const float Dx = gp.x - sp.x, Dy = gp.y - sp.y, Dz = gp.z - sp.z;
    const float ex = op.x - so.x, ey = op.y - so.y, ez = op.z - so.z;
    const float A = fmaf(Dx, Dx, fmaf(Dy, Dy, Dz * Dz));
    const float B = fmaf(ex, fmaf(2.0f, Dx, ex), fmaf(ey, fmaf(2.0f, Dy, ey), ez * fmaf(2.0f, Dz, ez)));
    const float s2 = A + B;
    const float rho = s2 > 0.0f ? rsqrtf(s2) : 0.0f;
    const float r0f = s2 * rho;
    const float e = fmaf(-r0f, r0f, A);
    const float c = (e + B) * (0.5f * rho);
    const float th = tau_hi * r0f;
    float te = fmaf(tau_hi, r0f, -th);
    te = fmaf(tau_hi, c, te);
    te = fmaf(tau_lo, r0f, te);
    const float f = (th - rintf(th)) + te;
    float sn, cs;
    __sincosf(6.28318530717958647692f * f, &sn, &cs);
    return mk<float>(cs * rho, sn * rho);
}

// 16 columns of tensor memory for this warp's 32 lanes (rows), added into v
__device__ __forceinline__ void t5_ld16_add(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] += __uint_as_float(r[i]);
}

// 32 columns of tensor memory for this warp's 32 lanes (rows), added into v
__device__ __forceinline__ void t5_ld32_add(uint32_t taddr, float* v) {
    t5_ld16_add(taddr, v);
    t5_ld16_add(taddr + 16, v + 16);
}

// 32 columns of tensor memory for this warp's 32 lanes set to v
__device__ __forceinline__ void t5_st32(uint32_t taddr, const float* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]),
        "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15]), "f"(v[16]),
        "f"(v[17]), "f"(v[18]), "f"(v[19]), "f"(v[20]), "f"(v[21]), "f"(v[22]), "f"(v[23]), "f"(v[24]),
        "f"(v[25]), "f"(v[26]), "f"(v[27]), "f"(v[28]), "f"(v[29]), "f"(v[30]), "f"(v[31]));
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Split charge operand B of every (source tile g, pass p) in the shared-memory layout:
// block (g, p) at blk + (g * npass + p) * kT5Blk, hi part then lo part, row r = right-hand side
// p * 64 + r, columns [Re q_j | Im q_j] over the tile's 16 sources.  Tile g covers sources
// tfirst[g] .. tfirst[g] + tn[g] - 1 (tn <= 16); absent sources and right-hand sides are zero.
// One block of 256 threads per (g, p); q: the sorted charges (nsrc, R) in float64.
__global__ void __launch_bounds__(256) k_t5_bsplit(const int32_t* __restrict__ tfirst, const int32_t* __restrict__ tn,
                                                   int ntiles, int npass, const cxd* __restrict__ q, int R,
                                                   unsigned char* __restrict__ blk) {
    const int64_t gp = blockIdx.x;
    if (gp >= (int64_t)ntiles * npass) return;
    const int g = (int)(gp / npass), p = (int)(gp % npass);
    const int f = tfirst[g], sn = tn[g];
    unsigned char* hi = blk + (size_t)gp * kT5Blk;
    unsigned char* lo = hi + kT5OpB;
    for (int e = threadIdx.x; e < kT5Rhs * (kT5K / 4); e += blockDim.x) {
        const int n = e % kT5Rhs, c = e / kT5Rhs;      // row fastest: coalesced charge reads
        const int r = p * kT5Rhs + n;
        float v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int k = 4 * c + i, j = k % kT5Src;
            float x = 0.f;
            if (j < sn && r < R) {
                const cxd z = q[(int64_t)(f + j) * R + r];
                x = k < kT5Src ? (float)z.x : (float)z.y;
            }
            v[i] = x;
        }
        t5_store4(hi, lo, t5_off(n, c, kT5SboB), v[0], v[1], v[2], v[3]);
    }
}

// Arguments of k_p2p_tc5.  A unit is (target box, first target of its 128-chunk, tiles over
// its neighbour list, 0); CTA c takes units cta_off[c] .. cta_off[c + 1] - 1 in order.
// stbase[s]: index of source box s's first tile in the B blocks.
struct T5Args {
    const int4* units;
    const int32_t* cta_off;
    const int32_t *tstart, *tcount, *sstart, *scount, *noff, *nidx, *stbase;
    const unsigned char* bblk;
    P2PMixedArgs a;
    cxd* phis;    // (nt, R) sorted: overwritten rows of every unit
    int R;
    int* err;     // set to 1 when a wait gave up (the result is then incomplete)
};

struct T5Ctl {
    uint64_t afull[kT5Stages], bfull[kT5Stages], empty[kT5Stages];
    uint64_t accfull[kT5Acc], accempty[kT5Acc];
    uint32_t tmem;
    int abort;
    int b_issued, b_used, mma_issued;
};

__global__ void __launch_bounds__(kT5Threads, 1) k_p2p_tc5(T5Args g) {
    extern __shared__ __align__(1024) unsigned char t5_smem[];
    __shared__ T5Ctl ctl;
    unsigned char* base = t5_smem + ((1024 - (smem_u32(t5_smem) & 1023)) & 1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int* abort = &ctl.abort;
    const int u0 = g.cta_off[blockIdx.x], u1 = g.cta_off[blockIdx.x + 1];
    const int npass = (g.R + kT5Rhs - 1) / kT5Rhs;
    if (tid == 0) {
        for (int s = 0; s < kT5Stages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&ctl.afull[s])), "r"(kT5Prod));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&ctl.bfull[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&ctl.empty[s])));
        }
        for (int a = 0; a < kT5Acc; ++a) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&ctl.accfull[a])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&ctl.accempty[a])), "r"(kT5Epi));
        }
        ctl.abort = 0;
        ctl.b_issued = ctl.b_used = ctl.mma_issued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == kT5Prod + kT5Epi) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl.tmem)),
                     "r"(kT5Cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = ctl.tmem;

    if (warp < kT5Prod) {
        // ---------------- producers: kernel values of row `row`, sources 8 h .. 8 h + 7 ----
        const int row = tid & (kT5M - 1), h = tid >> 7;
        int i = 0;   // tile counter of this CTA
        bool ok = true;
        for (int u = u0; u < u1 && ok; ++u) {
            const int4 un = g.units[u];
            const int b = un.x, c0 = un.y;
            const int t0 = g.tstart[b], tc = g.tcount[b];
            const bool active = c0 + row < tc;
            float4 gp = make_float4(0, 0, 0, 0), op = gp;
            if (active) {
                gp = g.a.tpt[t0 + c0 + row];
                op = g.a.tof[t0 + c0 + row];
            }
            for (int p = 0; p < npass && ok; ++p) {
                for (int nb = g.noff[b]; nb < g.noff[b + 1] && ok; ++nb) {
                    const int s = g.nidx[nb];
                    const int s0 = g.sstart[s], sc = g.scount[s], tb = g.stbase[s];
                    for (int sb = 0; sb < sc; sb += kT5Src, ++i) {
                        const int st = i % kT5Stages;
                        ok = t5_wait_ab(smem_u32(&ctl.empty[st]), ((i / kT5Stages) & 1) ^ 1, abort);
                        ok = __all_sync(0xffffffffu, ok);
                        if (!ok) break;
                        unsigned char* stage = base + st * kT5Stage;
                        if (tid == 0) {
                            const uint32_t fb = smem_u32(&ctl.bfull[st]);
                            const unsigned char* src = g.bblk + ((size_t)(tb + sb / kT5Src) * npass + p) * kT5Blk;
                            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                                         "r"((uint32_t)kT5Blk)
                                         : "memory");
                            asm volatile(
                                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
                                "[%3];" ::"r"(smem_u32(stage + 2 * kT5OpA)),
                                "l"(src), "r"((uint32_t)kT5Blk), "r"(fb)
                                : "memory");
                            ctl.b_issued = i + 1;
                        }
                        const int sn = min(kT5Src, sc - sb);
                        float re[8], imv[8];
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj) {
                            const int j = 8 * h + jj;
                            cxf v = mk<float>(0.f, 0.f);
                            if (active && j < sn) {
                                const float4 sp = __ldg(&g.a.spt[s0 + sb + j]);
                                const float4 so = __ldg(&g.a.sof[s0 + sb + j]);
                                v = t5_green(gp, op, sp, so, g.a.tau_hi, g.a.tau_lo);
                            }
                            re[jj] = v.x;
                            imv[jj] = v.y;
                        }
                        unsigned char* ahi = stage;
                        unsigned char* alo = stage + kT5OpA;
                        // Re G: chunks 2 h, 2 h + 1; Im G: 4 + 2 h, ...; -Im G: 8 + 2 h, ...
                        t5_store4(ahi, alo, t5_off(row, 2 * h, kT5SboA), re[0], re[1], re[2], re[3]);
                        t5_store4(ahi, alo, t5_off(row, 2 * h + 1, kT5SboA), re[4], re[5], re[6], re[7]);
                        t5_store4_pair(ahi, alo, t5_off(row, 4 + 2 * h, kT5SboA), t5_off(row, 8 + 2 * h, kT5SboA),
                                       imv);
                        t5_store4_pair(ahi, alo, t5_off(row, 5 + 2 * h, kT5SboA), t5_off(row, 9 + 2 * h, kT5SboA),
                                       imv + 4);
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        __syncwarp();
                        if (lane == 0) t5_arrive(smem_u32(&ctl.afull[st]));
                    }
                }
            }
        }
    } else if (warp < kT5Prod + kT5Epi) {
        // ---------------- epilogue: rows 32 q .. 32 q + 31, right-hand sides 32 e .. 32 e + 31 ----
        const int w = warp - kT5Prod, q = w & 3, e = w >> 2;
        const uint32_t lanes = (uint32_t)(32 * q) << 16;
        const int row = 32 * q + lane;
        float accr[32], acci[32];
        int i = 0;
        bool ok = true;
        for (int u = u0; u < u1 && ok; ++u) {
            const int4 un = g.units[u];
            const int b = un.x, c0 = un.y, nt = un.z;
            const int t0 = g.tstart[b], tc = g.tcount[b];
            for (int p = 0; p < npass && ok; ++p) {
#pragma unroll
                for (int k = 0; k < 32; ++k) accr[k] = acci[k] = 0.f;
                bool have_sum = false;
                for (int t = 0; t < nt; ++t, ++i) {
                    const int a = i % kT5Acc;
                    ok = t5_wait_ab(smem_u32(&ctl.accfull[a]), (i / kT5Acc) & 1, abort);
                    ok = __all_sync(0xffffffffu, ok);
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t col = tmem + lanes + (uint32_t)(a * kT5N + 32 * e);
                    t5_ld32_add(col, accr);
                    t5_ld32_add(col + kT5Rhs, acci);
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) t5_arrive(smem_u32(&ctl.accempty[a]));
                    if ((t + 1) % kT5Flush == 0 && t + 1 < nt) {
                        // registers into the block sums
                        const uint32_t sc = tmem + lanes + kT5SumCol + (uint32_t)(32 * e);
                        if (have_sum) {
                            t5_ld32_add(sc, accr);
                            t5_ld32_add(sc + kT5Rhs, acci);
                        }
                        t5_st32(sc, accr);
                        t5_st32(sc + kT5Rhs, acci);
#pragma unroll
                        for (int k = 0; k < 32; ++k) accr[k] = acci[k] = 0.f;
                        have_sum = true;
                    }
                }
                if (!ok) break;
                if (have_sum) {
                    const uint32_t sc = tmem + lanes + kT5SumCol + (uint32_t)(32 * e);
                    t5_ld32_add(sc, accr);
                    t5_ld32_add(sc + kT5Rhs, acci);
                }
                if (c0 + row < tc) {
                    const int r0 = p * kT5Rhs + 32 * e;
                    cxd* o = g.phis + (int64_t)(t0 + c0 + row) * g.R + r0;
                    const int rn = min(32, g.R - r0);
#pragma unroll
                    for (int k = 0; k < 32; ++k)
                        if (k < rn)
                            o[k] = mk<double>(f2d_bits(accr[k] * g.a.inv_unit_f), f2d_bits(acci[k] * g.a.inv_unit_f));
                }
            }
        }
    } else if (lane == 0) {
        // ---------------- MMA issue ----------------
        int i = 0;
        bool ok = true;
        for (int u = u0; u < u1 && ok; ++u) {
            const int nt = g.units[u].z;
            for (int p = 0; p < npass && ok; ++p)
                for (int t = 0; t < nt; ++t, ++i) {
                    const int st = i % kT5Stages, a = i % kT5Acc;
                    const uint32_t ph = (i / kT5Stages) & 1;
                    ok = t5_wait_ab(smem_u32(&ctl.bfull[st]), ph, abort);
                    if (ok) ctl.b_used = i + 1;
                    ok = ok && t5_wait_ab(smem_u32(&ctl.afull[st]), ph, abort);
                    ok = ok && t5_wait_ab(smem_u32(&ctl.accempty[a]), ((i / kT5Acc) & 1) ^ 1, abort);
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t s_a = smem_u32(base + st * kT5Stage);
                    const uint32_t ahi = s_a, alo = s_a + kT5OpA, bhi = s_a + 2 * kT5OpA, blo = bhi + kT5OpB;
                    const uint32_t d = tmem + (uint32_t)(a * kT5N);
                    // K step ks covers B chunks 2 ks, 2 ks + 1 (ks < 2: Re q, else Im q).  Re phi
                    // takes A chunks of Re G then -Im G, Im phi those of Im G then Re G.
#pragma unroll
                    for (int ks = 0; ks < kT5K / 8; ++ks) {
                        const uint32_t kb = (uint32_t)ks * 2u * kT5Lbo;
                        const uint32_t kre = (uint32_t)(ks < 2 ? 2 * ks : 8 + 2 * (ks - 2)) * kT5Lbo;
                        const uint32_t kim = (uint32_t)(ks < 2 ? 4 + 2 * ks : 2 * (ks - 2)) * kT5Lbo;
                        const uint64_t bh = t5_desc(bhi + kb, kT5SboB), bl = t5_desc(blo + kb, kT5SboB);
                        const uint32_t acc = ks > 0 ? 1u : 0u;
                        t5_mma(d, t5_desc(ahi + kre, kT5SboA), bh, acc);
                        t5_mma(d, t5_desc(ahi + kre, kT5SboA), bl, 1u);
                        t5_mma(d, t5_desc(alo + kre, kT5SboA), bh, 1u);
                        t5_mma(d + kT5Rhs, t5_desc(ahi + kim, kT5SboA), bh, acc);
                        t5_mma(d + kT5Rhs, t5_desc(ahi + kim, kT5SboA), bl, 1u);
                        t5_mma(d + kT5Rhs, t5_desc(alo + kim, kT5SboA), bh, 1u);
                    }
                    t5_commit(smem_u32(&ctl.empty[st]));
                    t5_commit(smem_u32(&ctl.accfull[a]));
                    ctl.mma_issued = i + 1;
                }
        }
    }
    __syncthreads();
    if (ctl.abort) {
        // drain what this CTA still has in flight before its shared and tensor memory go
        if (tid == 0) {
            for (int i = ctl.b_used; i < ctl.b_issued; ++i)
                t5_wait(smem_u32(&ctl.bfull[i % kT5Stages]), (i / kT5Stages) & 1);
            const int m = ctl.mma_issued;
            if (m > 0) t5_wait(smem_u32(&ctl.accfull[(m - 1) % kT5Acc]), ((m - 1) / kT5Acc) & 1);
            atomicExch(g.err, 1);
        }
        __syncthreads();
    }
    if (warp == kT5Prod + kT5Epi) {
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kT5Cols));
    }
}

// Watchdog self-test: one thread waits on an mbarrier that nothing completes, gives up after
// the bounded wait and sets the flag, exactly as the tcgen05 near field does.
__global__ void k_t5_watchdog_probe(int* __restrict__ err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    const uint32_t mb = smem_u32(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
    if (!t5_wait(mb, 0)) atomicExch(err, 1);
}

}  // namespace hfmm
