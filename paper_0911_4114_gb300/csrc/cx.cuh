// Complex arithmetic on interleaved (re, im) pairs, templated on the real type.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hfmm {

template <typename R>
struct alignas(2 * sizeof(R)) cx {
    R x, y;
};

template <typename R>
__host__ __device__ __forceinline__ cx<R> mk(R a, R b) {
    cx<R> c;
    c.x = a;
    c.y = b;
    return c;
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return mk<R>(a.x + b.x, a.y + b.y); }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return mk<R>(a.x - b.x, a.y - b.y); }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
    return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return mk<R>(s * a.x, s * a.y); }
template <typename R>
__host__ __device__ __forceinline__ cx<R> conj(cx<R> a) { return mk<R>(a.x, -a.y); }
// multiply by -i (forward) or +i (inverse)
template <typename R>
__host__ __device__ __forceinline__ cx<R> mul_mi(cx<R> a) { return mk<R>(a.y, -a.x); }
template <typename R>
__host__ __device__ __forceinline__ cx<R> mul_pi(cx<R> a) { return mk<R>(-a.y, a.x); }
// a += b * c
template <typename R>
__host__ __device__ __forceinline__ void mac(cx<R>& a, cx<R> b, cx<R> c) {
    a.x += b.x * c.x - b.y * c.y;
    a.y += b.x * c.y + b.y * c.x;
}
template <typename To, typename Ti>
__host__ __device__ __forceinline__ cx<To> cvt(cx<Ti> a) { return mk<To>((To)a.x, (To)a.y); }
// real scalar of type R from a double (works for float, double and double-float)
template <typename R>
__host__ __device__ __forceinline__ R rval(double v) { return (R)v; }

using cxd = cx<double>;
using cxf = cx<float>;

#ifdef __CUDACC__
// a / b as a real scalar of type R for positive integers a, b (FFT normalisations); float32:
// the correctly rounded quotient, without the float64 division (the slow float64 pipe)
template <typename R>
__device__ __forceinline__ R rratio(int a, int b) { return rval<R>((double)a / (double)b); }
template <>
__device__ __forceinline__ float rratio<float>(int a, int b) { return __fdiv_rn((float)a, (float)b); }

// read-only (non-coherent cache) load of a float64 complex value
__device__ __forceinline__ cxd ldg_cx(const cxd* p) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    return mk<double>(v.x, v.y);
}
#endif

}  // namespace hfmm
