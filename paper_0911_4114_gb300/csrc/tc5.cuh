// Float32 near field for many right-hand sides on the 5th-generation tensor cores
// (tcgen05.mma kind::tf32, accumulators in tensor memory), one persistent CTA per SM.
//
// The near-field sum phi_t,r = sum_s G(x_t, y_s) q_s,r over a target chunk's neighbour
// sources is, for a chunk of 128 targets, a complex GEMM.  Written as one real GEMM per tile
// of 16 sources,
//     C[t][n] = sum_k' A[t][k'] B[n][k'],   A = [Re G | Im G]           (128 x 32),
//     B[r][.] = [Re q_r | -Im q_r], B[64 + r][.] = [Im q_r | Re q_r]    (128 x 32, 64 RHS),
// so C[t][r] = Re phi and C[t][64 + r] = Im phi.  Each factor is split into two TF32 parts and
// three products (hi hi, hi lo, lo hi) accumulate in float32 (3xTF32), which keeps float32
// accuracy.  A is read by the MMAs from tensor memory (row t in lane t, one TF32 value per
// column), so neither its stores nor its reads take shared-memory bandwidth, which the MMAs'
// B reads and the charge copies need.  B is K-major with 128-byte rows (32 TF32 values) in the
// 128-byte swizzled shared-memory layout: row r at byte 128 r, its 16-byte chunk c at position
// c ^ (r mod 8), so the tensor core reads the 8 rows of a K step from 8 different bank groups.
//
// The charges do not depend on the target, so the split charges of every (source tile,
// 64-RHS pass), rows [Re q_r | Im q_r], are written once per apply into global memory in this
// layout (k_t5_bsplit, 16 KB per block) and brought by bulk asynchronous copies into the
// upper half of a B slot, which the producers then expand in place into the two row blocks of
// B (a sign change and a swap of halves): B's redundancy never crosses the memory system.  The
// kernel values A depend on both points and are computed in the CTA.  The CTA's warps have
// fixed roles around two tensor-memory A slots, six shared-memory B slots and two
// tensor-memory accumulators:
//   * 1 loader warp: walks the CTA's tile records (first source, count, charge block; read 32
//     at a time) and, as soon as a B slot is free, copies the tile's charges and its source
//     positions into it, up to six tiles ahead of the producers;
//   * 8 producer warps: for each tile wait for a free A slot and the tile's B slot, evaluate
//     the 128 x 16 kernel values of the exact-grid float32 form (two threads per target row,
//     8 sources each; branch-free, so a thread's eight evaluations interleave), split them,
//     store A hi / lo into tensor memory (tcgen05.st) and expand B;
//   * 1 MMA thread: when a tile's A and B are ready and an accumulator is free, issue the 12
//     MMAs (M = 128, N = 128, K = 8: four K steps of three products) into a fresh accumulator
//     and commit to the A slot's, the B slot's and the accumulator's barriers;
//   * 8 epilogue warps (two per 32-lane quarter of tensor memory, 32 right-hand sides each):
//     read each tile's sums (tcgen05.ld) into float32 registers and release the accumulator;
//     every 64 tiles the registers are added into a float32 block sum held in the last 128
//     columns of tensor memory, and at the end of a (target chunk, pass) the total is written
//     as float64.
// A fresh accumulator per tile keeps the tensor pipe's float32 accumulation short (12
// products; summed over 512 sources in one accumulator it measured 7e-6 relative).  Every wait
// gives up after about one second or when another thread of the CTA gave up: the CTA then
// records HFMM's timeout flag, waits (bounded again) for its own copies and MMAs in flight,
// frees its tensor memory and returns.
#pragma once
#include <stdint.h>

#include "cx.cuh"
#include "df.cuh"

namespace hfmm {

constexpr int kT5M = 128;          // targets per CTA tile (MMA M)
constexpr int kT5Src = 16;         // sources per tile (K = 32: real and imaginary parts)
constexpr int kT5Rhs = 64;         // right-hand sides per pass (MMA N = 128)
constexpr int kT5K = 2 * kT5Src;   // operand row: 32 TF32 values = 128 bytes
constexpr int kT5N = 2 * kT5Rhs;
// tensor memory (512 columns): accumulators at 0 and 128, A slots (hi: 32 columns, lo: 32)
// at 256 and 320, float32 block sums at 384
constexpr int kT5ASlots = 2;       // A (kernel values) ring in tensor memory
constexpr int kT5BSlots = 6;       // B (charges + source positions) ring, filled ahead by the loader
constexpr int kT5Acc = 2;          // tensor-memory accumulators of 128 columns
constexpr uint32_t kT5ACol = 256;     // A slot s: columns 256 + 64 s .. (hi), + 32 .. (lo)
constexpr uint32_t kT5SumCol = 384;   // float32 block sums: columns 384..511
constexpr uint32_t kT5Cols = 512;     // tensor-memory columns allocated
constexpr int kT5Flush = 64;       // tiles summed in registers between block-sum updates
constexpr int kT5Prod = 8, kT5Epi = 8;   // producer and epilogue warps, then the MMA and loader warps
constexpr int kT5MmaWarp = kT5Prod + kT5Epi, kT5LoadWarp = kT5MmaWarp + 1;
constexpr int kT5Threads = 32 * (kT5LoadWarp + 1);
constexpr size_t kT5Op = (size_t)kT5M * kT5K * 4;   // one operand part (16 KB)
constexpr size_t kT5Blk = kT5Op;                    // split charges (hi, lo: 64 rows each) of one (tile, pass)
constexpr size_t kT5Slot = 2 * kT5Op;               // hi and lo part of a B slot
constexpr size_t kT5PosBytes = 2 * kT5Src * 16;     // grid points then offsets (float4)
constexpr size_t kT5Smem = kT5BSlots * kT5Slot + kT5BSlots * kT5PosBytes + 1024;   // + alignment
constexpr unsigned long long kT5WaitNs = 1000000000ull;   // give up a wait after 1 s
constexpr uint32_t kT5SuspendNs = 100000;                 // longest suspension of one mbarrier test

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// shared-memory matrix descriptor of a K-major operand in the 128-byte swizzled layout:
// start >> 4 (bits 0-13), leading byte offset (unused by this layout; 16 >> 4) (16-29),
// stride byte offset 1024 >> 4 between 8-row groups (32-45), fixed 0b001 (46-48), base offset
// 0 (49-51: the operands start on 1024-byte boundaries and K steps move the start only
// within a 128-byte row), swizzle mode 2 = 128-byte (61-63)
__device__ __forceinline__ uint64_t t5_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

// instruction descriptor of kind::tf32: D float32 (bits 4-5 = 1), A and B TF32 (bits 7-9,
// 10-12 = 2), both K-major, N >> 3 (bits 17-22), M >> 4 (bits 24-28)
__host__ __device__ constexpr uint32_t t5_idesc() {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kT5N >> 3) << 17) | ((uint32_t)(kT5M >> 4) << 24);
}

__device__ __forceinline__ void t5_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(t5_idesc()), "r"(accumulate));
}

// the same with A in tensor memory (TMEM address of its first column)
__device__ __forceinline__ void t5_mma_ta(uint32_t tmem, uint32_t a_tmem, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem),
        "r"(a_tmem), "l"(b), "r"(t5_idesc()), "r"(accumulate));
}

// 8 consecutive columns of tensor memory for this warp's 32 lanes
__device__ __forceinline__ void t5_st8(uint32_t taddr, const uint32_t* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(v[0]),
                 "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

__device__ __forceinline__ void t5_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar));
}

// test the mbarrier phase; a thread whose phase is not complete is suspended until it
// completes or kT5SuspendNs pass (so waiting warps do not take issue slots from working ones)
__device__ __forceinline__ bool t5_try_wait(uint32_t mbar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(phase), "r"(kT5SuspendNs));
    return ok != 0;
}

// bounded wait for the mbarrier phase; false after about kT5WaitNs
__device__ __forceinline__ bool t5_wait(uint32_t mbar, uint32_t phase) {
    if (t5_try_wait(mbar, phase)) return true;
    const unsigned long long t0 = global_ns();
    while (!t5_try_wait(mbar, phase))
        if (global_ns() - t0 > kT5WaitNs) return false;
    return true;
}

// bounded wait that also gives up when another thread of the CTA has (*abort set); a wait
// that runs out of time sets *abort
__device__ __forceinline__ bool t5_wait_ab(uint32_t mbar, uint32_t phase, volatile int* abort) {
    if (t5_try_wait(mbar, phase)) return true;
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

__device__ __forceinline__ void t5_expect(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// bulk copy global -> shared (16-byte aligned addresses, a size that is a multiple of 16),
// completing `bytes` transactions on mbar
__device__ __forceinline__ void t5_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

__device__ __forceinline__ uint32_t t5_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// byte offset of 16-byte chunk c (TF32 values 4c .. 4c + 3) of row r in the 128-byte swizzled
// K-major layout (the operand starts on a 1024-byte boundary)
__host__ __device__ __forceinline__ uint32_t t5_off(int r, int c) {
    return (uint32_t)r * 128u + ((uint32_t)(c ^ (r & 7)) << 4);
}

// four values as TF32 hi and lo parts at offset `off` of the hi and lo operands
__device__ __forceinline__ void t5_store4(unsigned char* hi, unsigned char* lo, uint32_t off, float a, float b,
                                          float c, float d) {
    const uint32_t ha = t5_tf32(a), hb = t5_tf32(b), hc = t5_tf32(c), hd = t5_tf32(d);
    uint4 h = make_uint4(ha, hb, hc, hd);
    uint4 l = make_uint4(t5_tf32(a - __uint_as_float(ha)), t5_tf32(b - __uint_as_float(hb)),
                         t5_tf32(c - __uint_as_float(hc)), t5_tf32(d - __uint_as_float(hd)));
    *reinterpret_cast<uint4*>(hi + off) = h;
    *reinterpret_cast<uint4*>(lo + off) = l;
}

// float32 kernel value of the exact-grid form (as green_grid in kernels.cuh)
__device__ __forceinline__ cxf t5_green(float4 gp, float4 op, float4 sp, float4 so, float tau_hi, float tau_lo) {
    const float Dx = gp.x - sp.x, Dy = gp.y - sp.y, Dz = gp.z - sp.z;
    const float ex = op.x - so.x, ey = op.y - so.y, ez = op.z - so.z;
    const float A = fmaf(Dx, Dx, fmaf(Dy, Dy, Dz * Dz));
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
    const float x = 6.28318530717958647692f * ((th - rintf(th)) + te);
    float sn, cs;
    sincos_hw(x, &sn, &cs);
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

// Split charges of every (source tile g, pass p) in the swizzled shared-memory layout: block
// (g, p) at blk + (g * npass + p) * kT5Blk, 64 rows of hi parts then 64 rows of lo parts; row r
// is [Re q | Im q] of right-hand side p * 64 + r over the tile's 16 sources.  Tile g covers
// sources tfirst[g] .. tfirst[g] + tn[g] - 1 (tn <= 16); absent sources and right-hand sides
// are zero.  One block of 256 threads per (g, p); q: the sorted charges (nsrc, R) in float64.
__global__ void __launch_bounds__(256) k_t5_bsplit(const int32_t* __restrict__ tfirst, const int32_t* __restrict__ tn,
                                                   int ntiles, int npass, const cxd* __restrict__ q, int R,
                                                   unsigned char* __restrict__ blk) {
    const int64_t gp = blockIdx.x;
    if (gp >= (int64_t)ntiles * npass) return;
    const int g = (int)(gp / npass), p = (int)(gp % npass);
    const int f = tfirst[g], sn = tn[g];
    unsigned char* hi = blk + (size_t)gp * kT5Blk;
    unsigned char* lo = hi + kT5Blk / 2;
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
        t5_store4(hi, lo, t5_off(n, c), v[0], v[1], v[2], v[3]);
    }
}

// Arguments of k_p2p_tc5.  A unit is (target box, first target of its 128-chunk, number of
// tiles, 0); CTA c takes units cta_off[c] .. cta_off[c + 1] - 1 in order.  The tiles of unit u
// (its neighbour boxes' 16-source tiles in list order) are recs[rec_off[u] ..], each (first
// sorted source, tile index g + (count - 1) << 27); a pass p reads charge block g * npass + p.
struct T5Args {
    const int4* units;
    const int32_t* cta_off;
    const int32_t *tstart, *tcount, *rec_off;
    const int2* recs;
    const unsigned char* bblk;
    P2PMixedArgs a;
    cxd* phis;    // (nt, R) sorted: overwritten rows of every unit
    int R;
    int* err;     // set to 1 when a wait gave up (the result is then incomplete)
};

struct T5Ctl {
    uint64_t afull[kT5ASlots], aempty[kT5ASlots], bfull[kT5BSlots], bempty[kT5BSlots];
    uint64_t accfull[kT5Acc], accempty[kT5Acc];
    uint32_t tmem;
    int abort;
    int b_issued, mma_issued;
};

__global__ void __launch_bounds__(kT5Threads, 1) k_p2p_tc5(T5Args g) {
    extern __shared__ __align__(1024) unsigned char t5_smem[];
    __shared__ T5Ctl ctl;
    unsigned char* base = t5_smem + ((1024 - (smem_u32(t5_smem) & 1023)) & 1023);
    unsigned char* bslot = base;                                   // [kT5BSlots][hi, lo]
    float4* pos = reinterpret_cast<float4*>(base + kT5BSlots * kT5Slot);   // [kT5BSlots][32]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int* abort = &ctl.abort;
    const int u0 = g.cta_off[blockIdx.x], u1 = g.cta_off[blockIdx.x + 1];
    const int npass = (g.R + kT5Rhs - 1) / kT5Rhs;
    if (tid == 0) {
        for (int s = 0; s < kT5ASlots; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&ctl.afull[s])), "r"(kT5Prod));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&ctl.aempty[s])));
        }
        for (int s = 0; s < kT5BSlots; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&ctl.bfull[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&ctl.bempty[s])));
        }
        for (int a = 0; a < kT5Acc; ++a) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&ctl.accfull[a])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&ctl.accempty[a])), "r"(kT5Epi));
        }
        ctl.abort = 0;
        ctl.b_issued = ctl.mma_issued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == kT5MmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl.tmem)),
                     "r"(kT5Cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = ctl.tmem;

    if (warp == kT5LoadWarp) {
        // ---------------- loader: charges and positions of tile i into B slot i mod 4 ----------
        int i = 0;
        bool ok = true;
        for (int u = u0; u < u1 && ok; ++u) {
            const int nt = g.units[u].z, r0 = g.rec_off[u];
            for (int p = 0; p < npass && ok; ++p)
                for (int k0 = 0; k0 < nt && ok; k0 += 32) {
                    const int2 mine = k0 + lane < nt ? g.recs[r0 + k0 + lane] : make_int2(0, 0);
                    const int kn = min(32, nt - k0);
                    for (int k = 0; k < kn; ++k, ++i) {
                        const int src = __shfl_sync(0xffffffffu, mine.x, k);
                        const int gt = __shfl_sync(0xffffffffu, mine.y, k);
                        const int bs = i % kT5BSlots;
                        ok = t5_wait_ab(smem_u32(&ctl.bempty[bs]), ((i / kT5BSlots) & 1) ^ 1, abort);
                        ok = __all_sync(0xffffffffu, ok);
                        if (!ok) break;
                        if (lane == 0) {
                            const unsigned char* blk = g.bblk + ((size_t)(gt & ((1 << 27) - 1)) * npass + p) * kT5Blk;
                            unsigned char* b = bslot + bs * kT5Slot;
                            const uint32_t fb = smem_u32(&ctl.bfull[bs]);
                            const uint32_t pb = 16u * kT5Src;   // whole tiles (the arrays are padded)
                            t5_expect(fb, (uint32_t)kT5Blk + 2 * pb);
                            // hi rows into rows 64..127 of B hi, lo rows into rows 64..127 of B lo
                            t5_copy(smem_u32(b + kT5Op / 2), blk, (uint32_t)(kT5Blk / 2), fb);
                            t5_copy(smem_u32(b + kT5Op + kT5Op / 2), blk + kT5Blk / 2, (uint32_t)(kT5Blk / 2), fb);
                            t5_copy(smem_u32(pos + bs * 2 * kT5Src), g.a.spt + src, pb, fb);
                            t5_copy(smem_u32(pos + bs * 2 * kT5Src + kT5Src), g.a.sof + src, pb, fb);
                            ctl.b_issued = i + 1;
                        }
                    }
                }
        }
    } else if (warp < kT5Prod) {
        // ---------------- producers: kernel values of row `row`, sources 8 h .. 8 h + 7 ----
        const int row = tid & (kT5M - 1), h = tid >> 7;
        // B expansion: charge row r = [Re q | Im q] (copied to row 64 + r) becomes row r =
        // [Re q | -Im q] and row 64 + r = [Im q | Re q]; thread (k, r) moves chunks k, 4 + k of
        // that row in both parts (rows r and 64 + r share the swizzle, 64 rows lie 8 KB apart)
        const int xr = tid & (kT5Rhs - 1), xk = tid >> 6;
        const uint32_t xo_r = t5_off(kT5Rhs + xr, xk), xo_i = t5_off(kT5Rhs + xr, 4 + xk);
        int i = 0;
        bool ok = true;
        for (int u = u0; u < u1 && ok; ++u) {
            const int4 un = g.units[u];
            if (un.z == 0) continue;
            const int t0 = g.tstart[un.x], tc = g.tcount[un.x];
            const bool active = un.y + row < tc;
            const bool warp_rows = un.y + 32 * (warp & 3) < tc;   // some row of this warp is a target
            float4 gp = make_float4(0, 0, 0, 0), op = gp;
            if (active) {
                gp = g.a.tpt[t0 + un.y + row];
                op = g.a.tof[t0 + un.y + row];
            }
            for (int t = 0; t < npass * un.z; ++t, ++i) {
                const int as = i % kT5ASlots, bs = i % kT5BSlots;
                ok = t5_wait_ab(smem_u32(&ctl.aempty[as]), ((i / kT5ASlots) & 1) ^ 1, abort);
                ok = ok && t5_wait_ab(smem_u32(&ctl.bfull[bs]), (i / kT5BSlots) & 1, abort);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                const float4* sp = pos + bs * 2 * kT5Src;
                // a warp whose 32 rows all lie past the chunk's end (the short last chunk of a
                // box) leaves its A rows as they are: those rows' sums are never written, and
                // rows of a GEMM do not mix
                if (warp_rows) {
                    float re[8], imv[8];
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) {
                        // sources past the tile's end are the next points (or the zero padding):
                        // finite values that meet zero charges in B; rows past the chunk's end
                        // are finite too and never written
                        const int j = 8 * h + jj;
                        const cxf v = t5_green(gp, op, sp[j], sp[kT5Src + j], g.a.tau_hi, g.a.tau_lo);
                        re[jj] = v.x;
                        imv[jj] = v.y;
                    }
                    // lane `row` of A slot as: columns 8 h .. 8 h + 7 (real parts), 16 + 8 h ..
                    // (imaginary parts); the lo parts 32 columns further
                    uint32_t hr[8], hm[8], lr[8], lm[8];
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) {
                        hr[jj] = t5_tf32(re[jj]);
                        hm[jj] = t5_tf32(imv[jj]);
                        lr[jj] = t5_tf32(re[jj] - __uint_as_float(hr[jj]));
                        lm[jj] = t5_tf32(imv[jj] - __uint_as_float(hm[jj]));
                    }
                    const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + kT5ACol + (uint32_t)(64 * as + 8 * h);
                    t5_st8(ta, hr);
                    t5_st8(ta + 16, hm);
                    t5_st8(ta + 32, lr);
                    t5_st8(ta + 48, lm);
                }
                {   // expand B (while the tensor-memory stores complete)
                    unsigned char* bp = bslot + bs * kT5Slot;
                    const uint32_t sg = 0x80000000u;
#pragma unroll
                    for (int part = 0; part < 2; ++part, bp += kT5Op) {
                        const uint4 vr = *reinterpret_cast<const uint4*>(bp + xo_r);
                        const uint4 vi = *reinterpret_cast<const uint4*>(bp + xo_i);
                        *reinterpret_cast<uint4*>(bp + xo_r - kT5Op / 2) = vr;
                        *reinterpret_cast<uint4*>(bp + xo_i - kT5Op / 2) = make_uint4(vi.x ^ sg, vi.y ^ sg, vi.z ^ sg, vi.w ^ sg);
                        *reinterpret_cast<uint4*>(bp + xo_r) = vi;
                        *reinterpret_cast<uint4*>(bp + xo_i) = vr;
                    }
                }
                if (warp_rows) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) t5_arrive(smem_u32(&ctl.afull[as]));
            }
        }
    } else if (warp < kT5MmaWarp) {
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
        // ---------------- MMA issue (warp kT5MmaWarp) ----------------
        const uint64_t bdesc0 = t5_desc(smem_u32(bslot));   // B slot 0; slots and parts move its start
        int i = 0;
        bool ok = true;
        for (int u = u0; u < u1 && ok; ++u) {
            const int nt = g.units[u].z;
            for (int t = 0; t < npass * nt; ++t, ++i) {
                const int as = i % kT5ASlots, bs = i % kT5BSlots, a = i % kT5Acc;
                ok = t5_wait_ab(smem_u32(&ctl.afull[as]), (i / kT5ASlots) & 1, abort);
                ok = ok && t5_wait_ab(smem_u32(&ctl.accempty[a]), ((i / kT5Acc) & 1) ^ 1, abort);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t ahi = tmem + kT5ACol + (uint32_t)(64 * as), alo = ahi + 32;
                const uint64_t bh = bdesc0 + (uint64_t)((bs * kT5Slot) >> 4), bl = bh + (kT5Op >> 4);
                const uint32_t d = tmem + (uint32_t)(a * kT5N);
                // K step ks: A columns 8 ks .. 8 ks + 7, B bytes 32 ks .. 32 ks + 31 of every row
                // (2 ks in the descriptor's 16-byte start-address field)
#pragma unroll
                for (int ks = 0; ks < kT5K / 8; ++ks) {
                    t5_mma_ta(d, ahi + 8 * ks, bh + 2 * ks, ks > 0 ? 1u : 0u);
                    t5_mma_ta(d, ahi + 8 * ks, bl + 2 * ks, 1u);
                    t5_mma_ta(d, alo + 8 * ks, bh + 2 * ks, 1u);
                }
                t5_commit(smem_u32(&ctl.aempty[as]));
                t5_commit(smem_u32(&ctl.bempty[bs]));
                t5_commit(smem_u32(&ctl.accfull[a]));
                ctl.mma_issued = i + 1;
            }
        }
    }
    __syncthreads();
    if (ctl.abort) {
        // drain what this CTA still has in flight before its shared and tensor memory go: the
        // latest copy of every B slot, then the MMAs (their last commit covers all before it)
        if (tid == 0) {
            for (int i = max(0, ctl.b_issued - kT5BSlots); i < ctl.b_issued; ++i)
                t5_wait(smem_u32(&ctl.bfull[i % kT5BSlots]), (i / kT5BSlots) & 1);
            const int m = ctl.mma_issued;
            if (m > 0) t5_wait(smem_u32(&ctl.accfull[(m - 1) % kT5Acc]), ((m - 1) / kT5Acc) & 1);
            atomicExch(g.err, 1);
        }
        __syncthreads();
    }
    if (warp == kT5MmaWarp) {
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
