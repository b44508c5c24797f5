// Spherical Bessel functions j_n, y_n and integer-order Bessel functions J_n in float64,
// written from their three-term recurrences:
//   z_{n-1} + z_{n+1} = (2n+1)/x z_n        (j_n, y_n)
//   J_{n-1} + J_{n+1} = (2n/x) J_n
// y_n by the (stable) upward recurrence from y_0 = -cos x / x, y_1 = -cos x / x^2 - sin x / x;
// j_n and J_n by Miller's downward recurrence from a start index well above max(n, x),
// normalised with the closed forms j_0 = sin x / x, j_1 = sin x / x^2 - cos x / x (whichever
// is larger in magnitude) and with J_0 + 2 sum_k J_2k = 1 respectively.
#include <algorithm>
#include <cmath>
#include <vector>

#include "host_plan.hpp"

namespace hfmm {

static int miller_start(int nmax, double x) {
    double m = std::max((double)nmax, x) + 30.0 + 8.0 * std::cbrt(std::max(x, 1.0));
    int s = (int)m + 1;
    return s + (s & 1);  // even
}

void sph_jn_all(int nmax, double x, double* out) {
    if (x == 0.0) {
        out[0] = 1.0;
        for (int n = 1; n <= nmax; ++n) out[n] = 0.0;
        return;
    }
    int m = miller_start(nmax, x);
    std::vector<double> t(m + 2, 0.0);
    t[m + 1] = 0.0;
    t[m] = 1e-300;
    for (int n = m; n >= 1; --n) {
        t[n - 1] = (2.0 * n + 1.0) / x * t[n] - t[n + 1];
        if (std::fabs(t[n - 1]) > 1e250) {
            for (int k = n - 1; k <= m + 1; ++k) t[k] *= 1e-250;
        }
    }
    double j0 = std::sin(x) / x;
    double j1 = std::sin(x) / (x * x) - std::cos(x) / x;
    double scale = (std::fabs(j0) >= std::fabs(j1)) ? j0 / t[0] : j1 / t[1];
    for (int n = 0; n <= nmax; ++n) out[n] = t[n] * scale;
}

void sph_yn_all(int nmax, double x, double* out) {
    out[0] = -std::cos(x) / x;
    if (nmax >= 1) out[1] = -std::cos(x) / (x * x) - std::sin(x) / x;
    for (int n = 1; n < nmax; ++n) out[n + 1] = (2.0 * n + 1.0) / x * out[n] - out[n - 1];
}

void bessel_jn_all(int nmax, double x, double* out) {
    if (x == 0.0) {
        out[0] = 1.0;
        for (int n = 1; n <= nmax; ++n) out[n] = 0.0;
        return;
    }
    int m = miller_start(nmax, x);
    std::vector<double> t(m + 2, 0.0);
    t[m + 1] = 0.0;
    t[m] = 1e-300;
    for (int n = m; n >= 1; --n) {
        t[n - 1] = (2.0 * n) / x * t[n] - t[n + 1];
        if (std::fabs(t[n - 1]) > 1e250) {
            for (int k = n - 1; k <= m + 1; ++k) t[k] *= 1e-250;
        }
    }
    double s = t[0];
    for (int k = 2; k <= m; k += 2) s += 2.0 * t[k];
    double scale = 1.0 / s;
    for (int n = 0; n <= nmax; ++n) out[n] = t[n] * scale;
}

bool is_235(int64_t k) {
    if (k <= 0) return false;
    for (int64_t p : {2, 3, 5})
        while (k % p == 0) k /= p;
    return k == 1;
}

int64_t round_fft(int64_t n, int64_t mult) {
    int64_t k = std::max<int64_t>(1, (n + mult - 1) / mult);
    while (!is_235(k)) ++k;
    return mult * k;
}

}  // namespace hfmm
