// Float32 near field for many right-hand sides on the 5th-generation tensor cores
// (tcgen05.mma kind::tf32, accumulators in tensor memory).
//
// The near-field sum phi_t,r = sum_s G(x_t, y_s) q_s,r over a target chunk's neighbour
// sources is, for a chunk of 128 targets, a complex GEMM.  Written as one real GEMM per tile
// of 16 sources,
//     C[t][n] = sum_k' A[t][k'] B[n][k'],   A = [Re G | Im G]           (128 x 32),
//     B[r][.] = [Re q_r | -Im q_r], B[64 + r][.] = [Im q_r | Re q_r]    (128 x 32, 64 RHS),
// so C[t][r] = Re phi and C[t][64 + r] = Im phi.  Each factor is split into two TF32 parts and
// three products (hi hi, hi lo, lo hi) accumulate in float32 (3xTF32), which keeps float32
// accuracy.  The CTA's 128 threads compute the kernel values of their target row (the exact
// grid form of the float32 near field) and the charge rows, store both operands in shared
// memory in the canonical K-major layout without swizzle (8 x 16-byte core matrices; leading
// byte offset 128 between core matrices along K, stride byte offset 1024 between 8-row
// groups), and one thread issues the MMAs (M = 128, N = 128, K = 8 each) into one of two
// 128-column tensor-memory accumulators.  Completion is tracked by an mbarrier
// (tcgen05.commit); each tile's sums are read back (tcgen05.ld) and added in float32
// registers, and every 64 tiles (1024 sources) into the float64 result.  Every wait on the mbarrier gives up
// after about one second of wall time: the CTA then records HFMM's timeout flag, waits
// (bounded again) for its own MMAs, frees its tensor memory and returns.
#pragma once
#include <stdint.h>

#include "cx.cuh"
#include "df.cuh"

namespace hfmm {

constexpr int kT5M = 128;          // targets per CTA (MMA M)
constexpr int kT5Src = 16;         // sources per tile (K = 32: real and imaginary parts)
constexpr int kT5Rhs = 64;         // right-hand sides per pass (MMA N = 128)
constexpr int kT5K = 2 * kT5Src;
constexpr int kT5N = 2 * kT5Rhs;
constexpr int kT5Flush = 64;       // tiles summed in float32 registers between float64 flushes
constexpr uint32_t kT5Lbo = 128;   // bytes between core matrices along K
constexpr uint32_t kT5Sbo = (kT5K / 4) * 128;   // bytes between 8-row groups (1024)
constexpr size_t kT5Op = (size_t)kT5M * kT5K * 4;   // bytes of one operand part (16 KB)
constexpr size_t kT5Smem = 4 * kT5Op + 1024;        // A hi, A lo, B hi, B lo + alignment slack
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
__device__ __forceinline__ uint64_t t5_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(kT5Lbo >> 4) << 16) |
           ((uint64_t)(kT5Sbo >> 4) << 32) | (1ull << 46);
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

__device__ __forceinline__ uint32_t t5_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// byte offset of element (row, e) in a K-major operand of kT5K columns (no swizzle)
__device__ __forceinline__ uint32_t t5_off(int row, int chunk) {
    return (uint32_t)(row >> 3) * kT5Sbo + (uint32_t)chunk * kT5Lbo + (uint32_t)(row & 7) * 16u;
}

// one row of an operand, hi and lo parts (kT5K values)
__device__ __forceinline__ void t5_store_row(unsigned char* hi, unsigned char* lo, int row, const float* v) {
#pragma unroll
    for (int c = 0; c < kT5K / 4; ++c) {
        uint4 h, l;
        uint32_t* hp = &h.x;
        uint32_t* lp = &l.x;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float x = v[4 * c + i];
            const uint32_t xh = t5_tf32(x);
            hp[i] = xh;
            lp[i] = t5_tf32(x - __uint_as_float(xh));
        }
        *reinterpret_cast<uint4*>(hi + t5_off(row, c)) = h;
        *reinterpret_cast<uint4*>(lo + t5_off(row, c)) = l;
    }
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

// 32 columns of the accumulator for this warp's 32 lanes (rows)
__device__ __forceinline__ void t5_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// charges rounded to float32 once per apply (the float64 -> float32 conversion runs on the
// float64 pipe, which the per-tile loads of the near field must not touch)
__global__ void k_charges_f32(const cxd* __restrict__ q, int64_t n, cxf* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = mk<float>((float)q[i].x, (float)q[i].y);
}

// One CTA (128 threads) per (target box, 128-target chunk); qs: the charges in float32
// (k_charges_f32).  phis rows of the chunk are overwritten.  err: set to 1 when a wait gave up (the result is then incomplete).
// Each tile's MMAs write a fresh accumulator (the tensor pipe's float32 accumulation over
// many tiles loses accuracy: measured 7e-6 relative after 512 sources against 4e-7 per
// tile); two accumulators alternate, so the CUDA cores add tile i - 1's sums into their
// float32 registers while the MMAs of tile i run.  Every kT5Flush tiles the registers are
// added to the float64 rows.
__global__ void __launch_bounds__(128) k_p2p_tc5(
    const int2* __restrict__ units, int nunits, const int32_t* __restrict__ tstart,
    const int32_t* __restrict__ tcount, const int32_t* __restrict__ sstart, const int32_t* __restrict__ scount,
    const int32_t* __restrict__ noff, const int32_t* __restrict__ nidx, P2PMixedArgs a,
    const cxf* __restrict__ qs, cxd* __restrict__ phis, int R, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char t5_smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    __shared__ float4 shp[kT5Src], sho[kT5Src];
    const int u = blockIdx.x;
    if (u >= nunits) return;                                   // block-uniform
    unsigned char* base = t5_smem + ((1024 - (smem_u32(t5_smem) & 1023)) & 1023);
    unsigned char* a_hi = base;
    unsigned char* a_lo = base + kT5Op;
    unsigned char* b_hi = base + 2 * kT5Op;
    unsigned char* b_lo = base + 3 * kT5Op;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t mb = smem_u32(&mbar);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"((uint32_t)(2 * kT5N)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    const int b = units[u].x, c0 = units[u].y;
    const int t0 = tstart[b], tc = tcount[b];
    const bool active = c0 + tid < tc;
    float4 gp = make_float4(0, 0, 0, 0), op = gp;
    if (active) {
        gp = a.tpt[t0 + c0 + tid];
        op = a.tof[t0 + c0 + tid];
    }
    uint32_t phase = 0;
    bool inflight = false;
    bool my_abort = false;   // one of this thread's waits gave up
    bool aborted = false;    // some thread's did (block-uniform: from a barrier reduction)
    const uint32_t a_hi_s = smem_u32(a_hi), a_lo_s = smem_u32(a_lo), b_hi_s = smem_u32(b_hi), b_lo_s = smem_u32(b_lo);
    float accr[kT5Rhs], acci[kT5Rhs];   // this thread's row: float32 sums of the tiles since the last flush

    // wait for the MMAs in flight (their operands and accumulator are then free)
    auto wait_mma = [&]() {
        if (!inflight) return;
        if (!t5_wait(mb, phase)) my_abort = true;
        phase ^= 1u;
        inflight = false;
    };
    // add accumulator `slot` (after its MMAs completed) into the registers
    auto gather = [&](int slot) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t col = tmem + lane_base + (uint32_t)(slot * kT5N);
#pragma unroll
        for (int h = 0; h < kT5Rhs / 32; ++h) {
            float v[32];
            t5_ld32(col + (uint32_t)(32 * h), v);
#pragma unroll
            for (int i = 0; i < 32; ++i) accr[32 * h + i] += v[i];
            t5_ld32(col + (uint32_t)(kT5Rhs + 32 * h), v);
#pragma unroll
            for (int i = 0; i < 32; ++i) acci[32 * h + i] += v[i];
        }
    };
    // registers into the float64 rows (scaled to length units); `first` overwrites them
    auto flush = [&](int r0, bool first) {
        if (active) {
            const int rn = min(kT5Rhs, R - r0);
#pragma unroll
            for (int r = 0; r < kT5Rhs; ++r)
                if (r < rn) {
                    cxd& o = phis[(int64_t)(t0 + c0 + tid) * R + r0 + r];
                    const double x = a.inv_unit * (double)accr[r], y = a.inv_unit * (double)acci[r];
                    if (first) o = mk<double>(x, y);
                    else o = mk<double>(o.x + x, o.y + y);
                }
        }
#pragma unroll
        for (int r = 0; r < kT5Rhs; ++r) accr[r] = acci[r] = 0.f;
    };

    for (int r0 = 0; r0 < R; r0 += kT5Rhs) {
#pragma unroll
        for (int r = 0; r < kT5Rhs; ++r) accr[r] = acci[r] = 0.f;
        int tile = 0;          // tiles issued in this pass
        int since = 0;         // tiles gathered since the last flush
        bool first = true;     // the next flush overwrites the rows
        for (int nb = noff[b]; nb < noff[b + 1] && !aborted; ++nb) {
            const int s = nidx[nb];
            const int s0 = sstart[s], sc = scount[s];
            for (int sb = 0; sb < sc; sb += kT5Src) {
                const int sn = min(kT5Src, sc - sb);
                if (tid < kT5Src) {
                    shp[tid] = tid < sn ? a.spt[s0 + sb + tid] : make_float4(0, 0, 0, 0);
                    sho[tid] = tid < sn ? a.sof[s0 + sb + tid] : make_float4(0, 0, 0, 0);
                }
                aborted = __syncthreads_or(my_abort) != 0;       // block-uniform
                if (aborted) break;
                float rowa[kT5K], rowb[kT5K];
                // A row: kernel values of this thread's target against the tile's sources
#pragma unroll
                for (int j = 0; j < kT5Src; ++j) {
                    cxf g = mk<float>(0.f, 0.f);
                    if (active && j < sn) g = t5_green(gp, op, shp[j], sho[j], a.tau_hi, a.tau_lo);
                    rowa[j] = g.x;
                    rowa[kT5Src + j] = g.y;
                }
                // B row n = tid: right-hand side r = n mod 64, real (n < 64) or imaginary part
                {
                    const int r = tid % kT5Rhs;
                    const bool im = tid >= kT5Rhs;
#pragma unroll
                    for (int j = 0; j < kT5Src; ++j) {
                        float qr = 0.f, qi = 0.f;
                        if (j < sn && r0 + r < R) {
                            const cxf q = qs[(int64_t)(s0 + sb + j) * R + r0 + r];
                            qr = q.x;
                            qi = q.y;
                        }
                        rowb[j] = im ? qi : qr;
                        rowb[kT5Src + j] = im ? qr : -qi;
                    }
                }
                wait_mma();                                      // tile - 1 done: operands free
                t5_store_row(a_hi, a_lo, tid, rowa);
                t5_store_row(b_hi, b_lo, tid, rowb);
                asm volatile("fence.proxy.async.shared::cta;");
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncthreads();
                if (tid == 0) {
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t dcol = tmem + (uint32_t)((tile & 1) * kT5N);
#pragma unroll
                    for (int ks = 0; ks < kT5K / 8; ++ks) {
                        const uint32_t ko = (uint32_t)ks * 2u * kT5Lbo;
                        const uint64_t ah = t5_desc(a_hi_s + ko), al = t5_desc(a_lo_s + ko);
                        const uint64_t bh = t5_desc(b_hi_s + ko), bl = t5_desc(b_lo_s + ko);
                        t5_mma(dcol, ah, bh, ks > 0 ? 1u : 0u);
                        t5_mma(dcol, ah, bl, 1u);
                        t5_mma(dcol, al, bh, 1u);
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb));
                }
                inflight = true;
                if (tile > 0) {                                  // tile - 1's sums, beside tile's MMAs
                    gather((tile - 1) & 1);
                    if (++since == kT5Flush) {
                        flush(r0, first);
                        first = false;
                        since = 0;
                    }
                }
                ++tile;
            }
        }
        if (aborted) break;
        if (tile > 0) {
            wait_mma();
            gather((tile - 1) & 1);
        }
        flush(r0, first);                                        // also zero rows without sources
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
    }
    wait_mma();
    asm volatile("tcgen05.fence::before_thread_sync;");
    aborted = __syncthreads_or(my_abort) != 0;
    if (tid == 0 && aborted) atomicExch(err, 1);
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * kT5N)));
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
