// T^{s,LL} transfer tables computed on the device (Algorithm BMTF followed by the per-row phi
// anterpolation of Section 3.3.2), for the canonical transfer vectors a level's interaction
// lists use, then reflected into every used vector and stored in the level's precision.
// The same steps as the host planner (planner.cpp), in float64:
//   columns (vector, phi_p), p < N_phi^full / 2: sample 1/2 T at 2l+1 theta points (Legendre
//     series of Eq. TransferFn), DFT, convolve with the Fourier coefficients of |sin| (Section
//     3.2), truncate to |n| <= N_theta/2 - 1, evaluate at the N_theta rows; Eq. NumSphereSym
//     gives the column p + N_phi^full / 2 of the mirrored row;
//   rows (vector, theta_n), n <= N_theta/2: DFT of the N_phi^full samples, keep the band of
//     N_phi(theta_n), inverse DFT at N_phi(theta_n) points;
//   reflections (x -> -x, y -> -y, z -> -z, x <-> y) are index permutations of (n, m).
// One block per (vector, column) and per (vector, row); twiddles exp(-2 pi i t / n) are formed
// in shared memory by sincospi of the exact fraction 2t/n.
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "cx.cuh"
#include "df.cuh"
#include "host_plan.hpp"

namespace hfmm {
namespace {

constexpr int kTabBlock = 256;

__device__ __forceinline__ cxd cmul(cxd a, cxd b) { return mk<double>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ cxd cmulc(cxd a, cxd b) { return mk<double>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }

// w[t] = exp(-2 pi i t / n), t < n
__device__ void twiddles(cxd* w, int n) {
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        double sn, cs;
        sincospi(2.0 * (double)t / (double)n, &sn, &cs);
        w[t] = mk<double>(cs, -sn);
    }
}

// Fourier coefficient of |sin(theta)| (Section 3.2): 2 / (pi (1 - k^2)) for even k, 0 for odd
__device__ __forceinline__ double s_tilde(int k) {
    if (k & 1) return 0.0;
    const double d = (double)k;
    return 2.0 / (3.14159265358979323846 * (1.0 - d * d));
}

__device__ __forceinline__ int modi(long long a, int n) { return (int)(((a % n) + n) % n); }

// grid[(vector, row n <= half, column p)] (nfull columns), one block per (vector, column p < nfull/2)
__global__ void k_tsl_columns(int ell, int ntheta, int nfull, const cxd* __restrict__ coef,
                              const double* __restrict__ rhat, cxd* __restrict__ grid) {
    extern __shared__ unsigned char smem_raw[];
    const int m = 2 * ell + 1, half = ntheta / 2, b = ntheta / 2 - 1, ncol = nfull / 2;
    const int c = blockIdx.x / ncol, p = blockIdx.x % ncol;
    cxd* cf = reinterpret_cast<cxd*>(smem_raw);   // ell + 1
    cxd* wm = cf + (ell + 1);                     // m
    cxd* wt = wm + m;                             // ntheta
    cxd* samp = wt + ntheta;                      // m
    cxd* tf = samp + m;                           // m (frequencies -ell..ell)
    cxd* co = tf + m;                             // 2b + 1
    double* ra = reinterpret_cast<double*>(co + 2 * b + 1);   // ell: (2n+1)/(n+1)
    double* rb = ra + ell;                                    // ell: n/(n+1)
    for (int n = threadIdx.x; n <= ell; n += blockDim.x) cf[n] = coef[(size_t)c * (ell + 1) + n];
    for (int n = threadIdx.x; n < ell; n += blockDim.x) {
        ra[n] = (2.0 * n + 1.0) / (n + 1.0);
        rb[n] = (double)n / (n + 1.0);
    }
    twiddles(wm, m);
    twiddles(wt, ntheta);
    __syncthreads();
    const double rx = rhat[3 * c], ry = rhat[3 * c + 1], rz = rhat[3 * c + 2];
    double sp, cp;
    sincospi(2.0 * (double)p / (double)nfull, &sp, &cp);
    // 1/2 T at theta_j = 2 pi j / m, phi_p
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        double st, ct;
        sincospi(2.0 * (double)j / (double)m, &st, &ct);
        const double t = cp * st * rx + sp * st * ry + ct * rz;
        double p0 = 1.0, p1 = t;
        cxd acc = cf[0];
        if (ell >= 1) acc = acc + t * cf[1];
        for (int n = 1; n < ell; ++n) {
            const double p2 = ra[n] * t * p1 - rb[n] * p0;
            acc = acc + p2 * cf[n + 1];
            p0 = p1;
            p1 = p2;
        }
        samp[j] = 0.5 * acc;
    }
    __syncthreads();
    // theta coefficients of degree <= ell (exact on 2 ell + 1 samples)
    for (int f = threadIdx.x; f < m; f += blockDim.x) {
        const int fr = f - ell;
        cxd acc = mk<double>(0, 0);
        const int step = modi(fr, m);
        int t = 0;
        for (int j = 0; j < m; ++j) {
            acc = acc + cmul(samp[j], wm[t]);
            t += step;
            if (t >= m) t -= m;
        }
        tf[f] = (1.0 / (double)m) * acc;
    }
    __syncthreads();
    // convolution with the |sin| coefficients, truncated to |n| <= b (odd differences vanish)
    for (int i = threadIdx.x; i < 2 * b + 1; i += blockDim.x) {
        const int n = i - b;
        cxd acc = mk<double>(0, 0);
        const int f0 = ((n + ell) % 2 == 0) ? -ell : -ell + 1;
        for (int f = f0; f <= ell; f += 2) acc = acc + s_tilde(n - f) * tf[f + ell];
        co[i] = acc;
    }
    __syncthreads();
    // rows theta_n = 2 pi n / ntheta, mirrored into column p + nfull / 2 (Eq. NumSphereSym)
    cxd* g = grid + (size_t)c * (half + 1) * nfull;
    for (int n = threadIdx.x; n < ntheta; n += blockDim.x) {
        cxd acc = mk<double>(0, 0);
        int t = modi(-(long long)b * n, ntheta);
        for (int i = 0; i < 2 * b + 1; ++i) {
            acc = acc + cmulc(co[i], wt[t]);   // co * conj(w)
            t += n;
            if (t >= ntheta) t -= ntheta;
        }
        if (n <= half) g[(size_t)n * nfull + p] = acc;
        const int nn = (ntheta - n) % ntheta;
        if (nn <= half) g[(size_t)nn * nfull + p + nfull / 2] = acc;
    }
}

// canonical table out[(vector, K)] from the grid rows: one block per (vector, row n)
__global__ void k_tsl_rows(int nfull, int half, int64_t K, const int* __restrict__ nphi, const int64_t* __restrict__ off,
                           const cxd* __restrict__ grid, cxd* __restrict__ out) {
    extern __shared__ unsigned char smem_raw[];
    const int c = blockIdx.x / (half + 1), n = blockIdx.x % (half + 1);
    const int np = nphi[n];
    const int b = min((nfull + 1) / 2, (np + 1) / 2) - 1;
    cxd* wf = reinterpret_cast<cxd*>(smem_raw);   // nfull
    cxd* wn = wf + nfull;                          // np
    cxd* row = wn + np;                            // nfull
    cxd* spec = row + nfull;                       // 2b + 1
    twiddles(wf, nfull);
    twiddles(wn, np);
    const cxd* gr = grid + ((size_t)c * (half + 1) + n) * nfull;
    for (int j = threadIdx.x; j < nfull; j += blockDim.x) row[j] = gr[j];
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * b + 1; i += blockDim.x) {
        const int f = i - b;
        cxd acc = mk<double>(0, 0);
        const int step = modi(f, nfull);
        int t = 0;
        for (int j = 0; j < nfull; ++j) {
            acc = acc + cmul(row[j], wf[t]);
            t += step;
            if (t >= nfull) t -= nfull;
        }
        spec[i] = (1.0 / (double)nfull) * acc;
    }
    __syncthreads();
    cxd* o = out + (size_t)c * K + off[n];
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
        cxd acc = mk<double>(0, 0);
        int t = modi(-(long long)b * j, np);
        for (int i = 0; i < 2 * b + 1; ++i) {
            acc = acc + cmulc(spec[i], wn[t]);
            t += j;
            if (t >= np) t -= np;
        }
        o[j] = acc;
    }
}

template <typename T> __device__ __forceinline__ cx<T> store_as(cxd v);
template <> __device__ __forceinline__ cxf store_as<float>(cxd v) { return mk<float>((float)v.x, (float)v.y); }
template <> __device__ __forceinline__ cxd store_as<double>(cxd v) { return v; }
template <> __device__ __forceinline__ cx<df> store_as<df>(cxd v) { return mk<df>(df_from_double(v.x), df_from_double(v.y)); }

// table[slot][k] = canonical table of the slot's vector at the reflected index of k
template <typename T>
__global__ void k_tsl_reflect(int nslot, int half, int64_t K, const int* __restrict__ nphi,
                              const int64_t* __restrict__ off, const int32_t* __restrict__ row_of,
                              const int32_t* __restrict__ slot_canon, const int32_t* __restrict__ slot_flags,
                              const cxd* __restrict__ canon, cx<T>* __restrict__ table) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)nslot * K) return;
    const int s = (int)(i / K);
    const int64_t k = i % K;
    const int n = row_of[k];
    const int np = nphi[n];
    const int m = (int)(k - off[n]);
    const int fl = slot_flags[s];
    int nn = n, mm = m;
    if (fl & 1) mm = modi((long long)np / 2 - mm, np);
    if (fl & 2) mm = modi(-(long long)mm, np);
    if (fl & 4) nn = half - nn;
    if (fl & 8) mm = modi((long long)np / 4 - mm, np);
    table[i] = store_as<T>(canon[(size_t)slot_canon[s] * K + off[nn] + mm]);
}

struct DevBuf {
    std::vector<void*> ptrs;
    ~DevBuf() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <typename T>
    cudaError_t up(T** d, const std::vector<T>& h) {
        void* v = nullptr;
        cudaError_t e = cudaMalloc(&v, std::max<size_t>(1, h.size() * sizeof(T)));
        if (e != cudaSuccess) return e;
        ptrs.push_back(v);
        *d = static_cast<T*>(v);
        return h.empty() ? cudaSuccess : cudaMemcpy(v, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    }
    template <typename T>
    cudaError_t alloc(T** d, size_t n) {
        void* v = nullptr;
        cudaError_t e = cudaMalloc(&v, std::max<size_t>(1, n * sizeof(T)));
        if (e != cudaSuccess) return e;
        ptrs.push_back(v);
        *d = static_cast<T*>(v);
        return cudaSuccess;
    }
};

}  // namespace

std::string device_tables(const TableJob& job, const Quadrature& q, int store, void** out, size_t* bytes) {
    *out = nullptr;
    *bytes = 0;
    const int nc = job.ncanon(), nslot = (int)job.slot_canon.size();
    const int ell = job.ell, ntheta = q.ntheta, half = ntheta / 2, nfull = job.nfull;
    const int64_t K = q.K;
    if (nc == 0 || nslot == 0) return "";
    DevBuf tmp;
    cxd *coef = nullptr, *grid = nullptr, *canon = nullptr;
    double* rhat = nullptr;
    int* nphi = nullptr;
    int64_t* off = nullptr;
    int32_t *row_of = nullptr, *sc = nullptr, *sf = nullptr;
    std::vector<cxd> hc(job.coef.size());
    for (size_t i = 0; i < hc.size(); ++i) hc[i] = mk<double>(job.coef[i].real(), job.coef[i].imag());
    std::vector<int32_t> hrow((size_t)K);
    for (size_t n = 0; n + 1 < q.off.size(); ++n)
        for (int64_t k = q.off[n]; k < q.off[n + 1]; ++k) hrow[k] = (int32_t)n;
    cudaError_t e;
#define TCK(x)                                                                   \
    do {                                                                         \
        e = (x);                                                                 \
        if (e != cudaSuccess) return std::string(#x ": ") + cudaGetErrorString(e); \
    } while (0)
    TCK(tmp.up(&coef, hc));
    TCK(tmp.up(&rhat, job.rhat));
    TCK(tmp.up(&nphi, q.nphi));
    TCK(tmp.up(&off, q.off));
    TCK(tmp.up(&row_of, hrow));
    TCK(tmp.up(&sc, job.slot_canon));
    TCK(tmp.up(&sf, job.slot_flags));
    TCK(tmp.alloc(&grid, (size_t)nc * (half + 1) * nfull));
    TCK(tmp.alloc(&canon, (size_t)nc * K));
    TCK(cudaMemset(grid, 0, sizeof(cxd) * (size_t)nc * (half + 1) * nfull));
    const int m = 2 * ell + 1, b = ntheta / 2 - 1;
    const size_t smc = sizeof(cxd) * ((ell + 1) + m + ntheta + m + m + (2 * b + 1)) + sizeof(double) * 2 * ell;
    if (smc > 48 * 1024) TCK(cudaFuncSetAttribute(k_tsl_columns, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc));
    k_tsl_columns<<<nc * (nfull / 2), kTabBlock, smc>>>(ell, ntheta, nfull, coef, rhat, grid);
    TCK(cudaGetLastError());
    int maxnp = 0;
    for (int v : q.nphi) maxnp = std::max(maxnp, v);
    const size_t smr = sizeof(cxd) * (nfull + maxnp + nfull + (std::min((nfull + 1) / 2, (maxnp + 1) / 2) * 2));
    if (smr > 48 * 1024) TCK(cudaFuncSetAttribute(k_tsl_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr));
    k_tsl_rows<<<nc * (half + 1), kTabBlock, smr>>>(nfull, half, K, nphi, off, grid, canon);
    TCK(cudaGetLastError());
    const size_t elem = store == 0 ? sizeof(cxf) : (store == 1 ? sizeof(cxd) : sizeof(cx<df>));
    void* table = nullptr;
    TCK(cudaMalloc(&table, std::max<size_t>(1, elem * (size_t)nslot * K)));
    const int64_t total = (int64_t)nslot * K;
    const unsigned g = (unsigned)((total + kTabBlock - 1) / kTabBlock);
    if (store == 0)
        k_tsl_reflect<float><<<g, kTabBlock>>>(nslot, half, K, nphi, off, row_of, sc, sf, canon, (cxf*)table);
    else if (store == 1)
        k_tsl_reflect<double><<<g, kTabBlock>>>(nslot, half, K, nphi, off, row_of, sc, sf, canon, (cxd*)table);
    else
        k_tsl_reflect<df><<<g, kTabBlock>>>(nslot, half, K, nphi, off, row_of, sc, sf, canon, (cx<df>*)table);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(table);
        return std::string("device transfer tables: ") + cudaGetErrorString(e);
    }
#undef TCK
    *out = table;
    *bytes = elem * (size_t)nslot * K;
    return "";
}

}  // namespace hfmm
