// hfmm_direct_noalloc: the mixed-precision near-field sum without any device allocation.
//
// Some callers cannot call cudaMalloc: code inside a host framework's operator whose device
// memory may only come from the framework's own pool (an allocation behind the pool's back
// escapes its accounting and its memory limit), and code on a latency-critical path, where
// a device allocation is an implicit synchronisation point between streams.  Such callers
// cannot build a plan, because planning allocates.  This entry point serves them: the
// caller passes device inputs and outputs, and the only extra device memory it uses -- the
// point coordinates converted to the exact grid + fraction form of the mixed near-field
// arithmetic and the bounding box -- lives in one file-scope __device__ array of fixed size
// that every GPU loading this library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/hfmm.h"
#include "cx.cuh"
#include "host_plan.hpp"

using namespace hfmm;

namespace {

constexpr int64_t kMaxPoints = HFMM_NOALLOC_MAX_POINTS;   // sources + targets
constexpr size_t kHeader = 256;                           // bounding box (6 doubles), padded
constexpr size_t kScratchBytes = kHeader + (size_t)kMaxPoints * 2 * sizeof(float4);
constexpr int kThreads = 128;
constexpr int kMaxDevices = 64;

// The scratch shared by every call on a device.  In host code this name is only a
// host-side stand-in: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

hfmm_status fail(hfmm_status s, const std::string& m) {
    hfmm::set_last_error(m);
    return s;
}

// bounding box of all points: one block, overwrites the six header doubles every call
__global__ void k_bbox(const double* __restrict__ s, int64_t ns, const double* __restrict__ t, int64_t nt,
                       double* __restrict__ box) {
    __shared__ double lo[3][kThreads], hi[3][kThreads];
    double l[3] = {INFINITY, INFINITY, INFINITY}, h[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = threadIdx.x; i < ns + nt; i += blockDim.x) {
        const double* p = (i < ns) ? s + 3 * i : t + 3 * (i - ns);
        for (int k = 0; k < 3; ++k) {
            l[k] = fmin(l[k], p[k]);
            h[k] = fmax(h[k], p[k]);
        }
    }
    for (int k = 0; k < 3; ++k) {
        lo[k][threadIdx.x] = l[k];
        hi[k][threadIdx.x] = h[k];
    }
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 3; ++k) {
                lo[k][threadIdx.x] = fmin(lo[k][threadIdx.x], lo[k][threadIdx.x + w]);
                hi[k][threadIdx.x] = fmax(hi[k][threadIdx.x], hi[k][threadIdx.x + w]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) {
            box[k] = lo[k][0];
            box[3 + k] = hi[k][0];
        }
}

// root cube of the bounding box (as the planner forms it, without contractions), then
// (grid integer, fraction) per coordinate on a 2^10 grid
__device__ void root_cube(const double* box, double corner[3], double* scale, double* side_out) {
    double side = fmax(__dadd_rn(box[3], -box[0]), fmax(__dadd_rn(box[4], -box[1]), __dadd_rn(box[5], -box[2])));
    if (side == 0.0) side = 1.0;
    for (int k = 0; k < 3; ++k) corner[k] = __dadd_rn(__dmul_rn(__dadd_rn(box[k], box[3 + k]), 0.5), -__dmul_rn(side, 0.5));
    *scale = __ddiv_rn(1024.0, side);
    *side_out = side;
}

__global__ void k_grid(const double* __restrict__ pts, int64_t n, const double* __restrict__ box,
                       float4* __restrict__ g, float4* __restrict__ o) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double corner[3], scale, side;
    root_cube(box, corner, &scale, &side);
    float gv[3], ov[3];
    for (int k = 0; k < 3; ++k) {
        double u = __dmul_rn(__dadd_rn(pts[3 * i + k], -corner[k]), scale);
        double f = fmin(fmax(floor(u), 0.0), 1023.0);
        gv[k] = (float)f;
        ov[k] = (float)__dadd_rn(u, -f);
    }
    g[i] = make_float4(gv[0], gv[1], gv[2], 0.f);
    o[i] = make_float4(ov[0], ov[1], ov[2], 0.f);
}

// every target against every source, same arithmetic as the planned mixed near field
template <typename T>
__global__ void k_direct(const float4* __restrict__ tg, const float4* __restrict__ to, int64_t nt,
                         const float4* __restrict__ sg, const float4* __restrict__ so, int64_t ns,
                         const cx<T>* __restrict__ q, cx<T>* __restrict__ phi, int R, const double* __restrict__ box,
                         double kappa) {
    __shared__ float4 shp[kThreads], sho[kThreads];
    __shared__ cxf shq[kThreads * 4];
    double corner[3], scale, side;
    root_cube(box, corner, &scale, &side);
    const double tau = __ddiv_rn(__dmul_rn(kappa, __ddiv_rn(side, 1024.0)), 2.0 * 3.14159265358979323846);
    const float tau_hi = (float)tau, tau_lo = (float)(tau - (double)tau_hi);
    const float two_pi = 6.28318530717958647692f;
    const int64_t ti = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool active = ti < nt;
    float4 gp = make_float4(0, 0, 0, 0), op = gp;
    if (active) {
        gp = tg[ti];
        op = to[ti];
    }
    for (int r0 = 0; r0 < R; r0 += 4) {
        const int rn = min(4, R - r0);
        cxd acc[4];
        for (int r = 0; r < 4; ++r) acc[r] = mk<double>(0, 0);
        for (int64_t sb = 0; sb < ns; sb += kThreads) {
            const int sn = (int)min((int64_t)kThreads, ns - sb);
            __syncthreads();
            if (threadIdx.x < sn) {
                shp[threadIdx.x] = sg[sb + threadIdx.x];
                sho[threadIdx.x] = so[sb + threadIdx.x];
                for (int r = 0; r < rn; ++r) shq[threadIdx.x * 4 + r] = cvt<float>(q[(sb + threadIdx.x) * R + r0 + r]);
            }
            __syncthreads();
            if (!active) continue;
            cxf tile[4];
            for (int r = 0; r < 4; ++r) tile[r] = mk<float>(0, 0);
            for (int jj = 0; jj < sn; ++jj) {
                const float4 sp = shp[jj], sq = sho[jj];
                const float Dx = gp.x - sp.x, Dy = gp.y - sp.y, Dz = gp.z - sp.z;
                const float ex = op.x - sq.x, ey = op.y - sq.y, ez = op.z - sq.z;
                const float A = fmaf(Dx, Dx, fmaf(Dy, Dy, Dz * Dz));
                const float B = fmaf(ex, fmaf(2.0f, Dx, ex), fmaf(ey, fmaf(2.0f, Dy, ey), ez * fmaf(2.0f, Dz, ez)));
                const float s2 = A + B;
                if (s2 <= 0.0f) continue;
                const float rho = rsqrtf(s2);
                const float r0f = s2 * rho;
                const float e = fmaf(-r0f, r0f, A);
                const float c = (e + B) * (0.5f * rho);
                const float th = tau_hi * r0f;
                float te = fmaf(tau_hi, r0f, -th);
                te = fmaf(tau_hi, c, te);
                te = fmaf(tau_lo, r0f, te);
                const float f = (th - rintf(th)) + te;
                float sn_, cs_;
                __sincosf(two_pi * f, &sn_, &cs_);
                const cxf gk = mk<float>(cs_ * rho, sn_ * rho);
                for (int r = 0; r < rn; ++r) mac(tile[r], gk, shq[jj * 4 + r]);
            }
            for (int r = 0; r < rn; ++r) {
                acc[r].x += (double)tile[r].x;
                acc[r].y += (double)tile[r].y;
            }
        }
        if (active)
            for (int r = 0; r < rn; ++r) phi[ti * R + r0 + r] = cvt<T>(scale * acc[r]);
    }
}

// first call on a device (with that device current): resolve the array's device address
hfmm_status scratch_for(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(HFMM_ERR_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return fail(HFMM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    return HFMM_OK;
}

}  // namespace

extern "C" {

hfmm_status hfmm_direct_noalloc(const double* sources, int64_t ns, const double* targets, int64_t nt,
                                const void* q, void* phi, int nrhs, hfmm_dtype dtype, double kappa,
                                void* stream) {
    if (!sources || !targets || !q || !phi) return fail(HFMM_ERR_ARG, "NULL pointer");
    if (ns < 1 || nt < 1) return fail(HFMM_ERR_ARG, "need ns >= 1 and nt >= 1");
    if (ns + nt > kMaxPoints)
        return fail(HFMM_ERR_ARG, "ns + nt = " + std::to_string(ns + nt) + " exceeds the static scratch limit of " +
                                      std::to_string(kMaxPoints) + " points");
    if (nrhs < 1 || nrhs > 4096) return fail(HFMM_ERR_ARG, "nrhs must be in [1, 4096]");
    if (dtype != HFMM_C64 && dtype != HFMM_C128) return fail(HFMM_ERR_ARG, "unknown dtype");
    if (!(kappa > 0.0)) return fail(HFMM_ERR_ARG, "kappa must be > 0");
    // an error left by earlier, unrelated work is reported as such and not cleared, so that
    // the caller's own error state survives and the launch check below sees only our launches
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess)
        return fail(HFMM_ERR_CUDA, std::string("a CUDA error was pending before hfmm_direct_noalloc was called "
                                               "(left in place): ") + cudaGetErrorString(e));
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(HFMM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    unsigned char* base = nullptr;
    hfmm_status s = scratch_for(dev, &base);
    if (s != HFMM_OK) return s;
    double* box = reinterpret_cast<double*>(base);
    float4* tg = reinterpret_cast<float4*>(base + kHeader);
    float4* to = tg + nt;
    float4* sg = to + nt;
    float4* so = sg + ns;
    cudaStream_t st = (cudaStream_t)stream;
    k_bbox<<<1, kThreads, 0, st>>>(sources, ns, targets, nt, box);
    k_grid<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(targets, nt, box, tg, to);
    k_grid<<<(unsigned)((ns + 255) / 256), 256, 0, st>>>(sources, ns, box, sg, so);
    const unsigned nb = (unsigned)((nt + kThreads - 1) / kThreads);
    if (dtype == HFMM_C64)
        k_direct<float><<<nb, kThreads, 0, st>>>(tg, to, nt, sg, so, ns, (const cxf*)q, (cxf*)phi, nrhs, box, kappa);
    else
        k_direct<double><<<nb, kThreads, 0, st>>>(tg, to, nt, sg, so, ns, (const cxd*)q, (cxd*)phi, nrhs, box, kappa);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HFMM_ERR_CUDA, std::string("hfmm_direct_noalloc launch: ") + cudaGetErrorString(e));
    return HFMM_OK;
}

}  // extern "C"
