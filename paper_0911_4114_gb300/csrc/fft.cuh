// Warp-level Fourier re-sampling in shared memory (Section 3.4 primitive).
//
// A length-n sequence is moved to length n' by a forward FFT, keeping the frequencies
// |k| <= min(ceil(n/2), ceil(n'/2)) - 1 (scaled by 1/n), and an inverse FFT of length n'
// (zero padding = interpolation, truncation = anterpolation).  Lengths factor into 2, 3
// and 5; the FFTs are self-sorting mixed-radix Stockham passes (radices 4, 2, 3, 5) over
// two shared-memory buffers owned by one warp, with twiddles exp(-2 pi i t / n) read
// from a per-length table.
#pragma once
#include "cx.cuh"
#include "df.cuh"

namespace hfmm {

struct TwiddleView {
    const void* pool;     // cx<R> tables, one per length, back to back
    const int* off;       // off[n] = first entry of the length-n table, -1 if absent
};

template <typename R>
__device__ __forceinline__ void dft_small(cx<R>* v, int radix, bool inv) {
    if (radix == 2) {
        cx<R> a = v[0], b = v[1];
        v[0] = a + b;
        v[1] = a - b;
    } else if (radix == 4) {
        cx<R> t0 = v[0] + v[2], t1 = v[0] - v[2], t2 = v[1] + v[3], t3 = v[1] - v[3];
        t3 = inv ? mul_pi(t3) : mul_mi(t3);
        v[0] = t0 + t2;
        v[2] = t0 - t2;
        v[1] = t1 + t3;
        v[3] = t1 - t3;
    } else if (radix == 3) {
        const R h = rval<R>(0.86602540378443864676);  // sqrt(3)/2
        cx<R> s = v[1] + v[2], d = v[1] - v[2];
        cx<R> m = v[0] - rval<R>(0.5) * s;
        cx<R> rot = inv ? mul_pi(h * d) : mul_mi(h * d);
        v[0] = v[0] + s;
        v[1] = m + rot;
        v[2] = m - rot;
    } else {  // radix 5
        const R c1 = rval<R>(0.30901699437494742410);   // cos(2 pi / 5)
        const R c2 = rval<R>(-0.80901699437494742410);  // cos(4 pi / 5)
        const R s1 = rval<R>(0.95105651629515357212);   // sin(2 pi / 5)
        const R s2 = rval<R>(0.58778525229247312917);   // sin(4 pi / 5)
        cx<R> a1 = v[1] + v[4], b1 = v[1] - v[4], a2 = v[2] + v[3], b2 = v[2] - v[3];
        cx<R> p1 = v[0] + c1 * a1 + c2 * a2;
        cx<R> p2 = v[0] + c2 * a1 + c1 * a2;
        cx<R> q1 = s1 * b1 + s2 * b2;
        cx<R> q2 = s2 * b1 - s1 * b2;
        q1 = inv ? mul_pi(q1) : mul_mi(q1);
        q2 = inv ? mul_pi(q2) : mul_mi(q2);
        v[0] = v[0] + a1 + a2;
        v[1] = p1 + q1;
        v[4] = p1 - q1;
        v[2] = p2 + q2;
        v[3] = p2 - q2;
    }
}

__device__ __forceinline__ int next_radix(int m) {
    if ((m & 3) == 0) return 4;
    if ((m & 1) == 0) return 2;
    if (m % 3 == 0) return 3;
    return 5;
}

// In-place-by-ping-pong FFT of a[0..n) (sign -1 forward, +1 inverse, unnormalised).
// Returns the buffer (a or b) that holds the result.  All 32 lanes must call it.
// Stage with ns accumulated outputs: element j = k + ns * g (k < ns) of each of the radix
// input strides is multiplied by exp(-+2 pi i k r / (ns radix)) = tw[k r n / (ns radix)],
// an index below n; r = 0 and the whole first stage (k = 0) have unit twiddles and skip it.
template <typename R>
__device__ cx<R>* warp_fft(cx<R>* a, cx<R>* b, int n, bool inv, const cx<R>* tw, int lane) {
    cx<R>* src = a;
    cx<R>* dst = b;
    int ns = 1, rest = n;
    while (rest > 1) {
        const int radix = next_radix(rest);
        const int nr = n / radix;
        const int stride = rest / radix;     // n / (ns * radix)
        // k = j mod ns through a float quotient: j, ns <= 1024, so j / ns is within 2^-14
        // of its value and the fractional parts are multiples of 1/ns >= 2^-10; adding
        // 2^-12 before truncation gives the exact floor
        const float inv_ns = 1.0f / (float)ns;
        for (int j = lane; j < nr; j += 32) {
            const int k = (ns == 1) ? 0 : j - ns * (int)fmaf((float)j, inv_ns, 0.000244140625f);
            cx<R> v[5];
            v[0] = src[j];
            if (ns == 1) {
                for (int r = 1; r < radix; ++r) v[r] = src[j + r * nr];
            } else {
                for (int r = 1; r < radix; ++r) {
                    cx<R> w = tw[k * r * stride];
                    if (inv) w = conj(w);
                    v[r] = src[j + r * nr] * w;
                }
            }
            dft_small(v, radix, inv);
            const int d = (j - k) * radix + k;
            for (int r = 0; r < radix; ++r) dst[d + r * ns] = v[r];
        }
        __syncwarp();
        cx<R>* t = src;
        src = dst;
        dst = t;
        ns *= radix;
        rest /= radix;
    }
    return src;
}

// Re-sample a[0..n) to length np; returns the buffer holding the np results.
template <typename R>
__device__ cx<R>* warp_resample(cx<R>* a, cx<R>* b, int n, int np, const TwiddleView& tv, int lane) {
    const cx<R>* pool = reinterpret_cast<const cx<R>*>(tv.pool);
    cx<R>* s = warp_fft(a, b, n, false, pool + tv.off[n], lane);
    cx<R>* o = (s == a) ? b : a;
    const int band = min((n + 1) / 2, (np + 1) / 2) - 1;
    const R scale = rratio<R>(1, n);
    for (int j = lane; j < np; j += 32) {
        int f = (2 * j <= np) ? j : j - np;
        cx<R> v = mk<R>(rval<R>(0.0), rval<R>(0.0));
        if (f <= band && f >= -band) v = scale * s[(f + n) % n];
        o[j] = v;
    }
    __syncwarp();
    return warp_fft(o, s, np, true, pool + tv.off[np], lane);
}

}  // namespace hfmm
