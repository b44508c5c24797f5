// Host planner of the Fourier-basis FMM (float64):
//   * octree over sources and targets, interaction lists and neighbour lists (Section 2);
//   * per level: truncation l (Eq. EBF start, Eq. CollinoError refinement, Section 2.1),
//     N_theta (Algorithm Ntheta), N_phi(theta_n) (Algorithm Nphi), the choice of alpha and
//     precision by the round-off estimate of the quadrature sum;
//   * T^{s,LL} for the canonical transfer vectors with x >= y >= 0, z >= 0 (Figure
//     SemiOctant) by Algorithm BMTF followed by the per-row phi anterpolation of Section
//     3.3.2, then reflected into the other vectors by index permutations (one buffer box:
//     34 canonical of 316; two buffer boxes, Section 3.3.3: 108 of 1206); only vectors that
//     the level's interaction lists use are computed.
//
// Conventions that the paper leaves open (identical rules are applied by the test oracle,
// which is an independent implementation):
//   root cube = given, or the bounding cube of all points (side = largest extent);
//   box index at depth D = clamp(floor((x - corner) * (2^D / side)), 0, 2^D - 1);
//   Morton order with the x bit above y above z; points by key then original index;
//   eps_l = eps_scale * eps, absolute threshold eps_l / |r0|, d0 = -log10(eps_l);
//   |r| = alpha sqrt(3) a_l, |r0| = (b + 1) a_l for b buffer boxes; N^max = 2l + 64 doubled
//   on failure;
//   N_theta rounded up to 2 * 2^a 3^b 5^c, N_phi to 4 * 2^a 3^b 5^c; rows mirrored about
//   theta = pi/2; re-sampling keeps |k| <= min(ceil(K/2), ceil(K'/2)) - 1.
// Built with -ffp-contract=off so the tree arithmetic rounds exactly as written.
#include <algorithm>
#include <cmath>
#include <parallel/algorithm>
#include <cstring>
#include <numeric>
#include <stdexcept>

#include "host_plan.hpp"

namespace hfmm {

static const double kPi = 3.14159265358979323846;
static const double kTwoPi = 2.0 * kPi;
static const double kFourPi2 = 4.0 * kPi * kPi;
// smallest kappa a_l of an active level: one buffer box needs boxes of about a wavelength
// (the Gegenbauer series converges only geometrically, ratio up to alpha sqrt(3)/2, for
// pairs near opposite corners of small boxes); with two buffer boxes the ratio is at most
// alpha sqrt(3)/3 and the round-off rule alone decides
static double min_ka(int buffer) { return buffer >= 2 ? 0.0 : 6.0; }

void Quadrature::finalize() {
    off.assign(nphi.size() + 1, 0);
    for (size_t n = 0; n < nphi.size(); ++n) off[n + 1] = off[n] + nphi[n];
    K = off.back();
}

// ---------------------------------------------------------------------------
// small DFT helpers: exact index reduction, twiddles from one cos/sin table
// ---------------------------------------------------------------------------
struct Twiddle {
    int n;
    std::vector<cd> w;  // w[t] = exp(-2 pi i t / n)
    explicit Twiddle(int n_) : n(n_), w(n_) {
        for (int t = 0; t < n; ++t) {
            double ang = kTwoPi * (double)t / (double)n;
            w[t] = cd(std::cos(ang), -std::sin(ang));
        }
    }
    // exp(-2 pi i a b / n) for integer a, b (any sign)
    cd fwd(int64_t a, int64_t b) const {
        int64_t t = ((a * b) % n + n) % n;
        return w[t];
    }
    cd inv(int64_t a, int64_t b) const { return std::conj(fwd(a, b)); }
};

static inline int mod(int64_t a, int64_t n) { return (int)(((a % n) + n) % n); }

// Fourier coefficient of |sin(theta)| (Section 3.2)
static double s_tilde(int64_t n) {
    if (n & 1) return 0.0;
    double d = (double)n;
    return 2.0 / (kPi * (1.0 - d * d));
}

// ---------------------------------------------------------------------------
// truncation (Section 2.1)
// ---------------------------------------------------------------------------
static void hankel_all(int nmax, double x, std::vector<cd>& h) {
    std::vector<double> j(nmax + 1), y(nmax + 1);
    sph_jn_all(nmax, x, j.data());
    sph_yn_all(nmax, x, y.data());
    h.resize(nmax + 1);
    for (int n = 0; n <= nmax; ++n) h[n] = cd(j[n], y[n]);
}

static double collino(int ell, double kappa, double r, double r0) {
    std::vector<cd> h;
    hankel_all(ell + 1, kappa * r0, h);
    std::vector<double> j(ell + 2);
    sph_jn_all(ell + 1, kappa * r, j.data());
    double best = 0.0;
    for (int s = 0; s < 2; ++s) {
        double sg = s == 0 ? 1.0 : -1.0;
        cd br = h[ell + 1] * j[ell] + sg * h[ell] * j[ell + 1];
        double v = kappa * kappa * (r * r0 / (r0 + sg * r)) * std::abs(br);
        best = std::max(best, v);
    }
    return best;
}

static int choose_ell(double kappa, double r, double r0, double eps_abs, double d0) {
    double kr = kappa * r;
    int l = (int)std::ceil(kr + 1.8 * std::pow(d0, 2.0 / 3.0) * std::cbrt(kr));
    l = std::max(1, l);
    auto pass = [&](int ll) { return collino(ll, kappa, r, r0) <= eps_abs; };
    if (pass(l)) {
        while (l > 1 && pass(l - 1)) --l;
    } else {
        int start = l;
        while (!pass(l)) {
            ++l;
            if (l > start + 2000) throw std::runtime_error("truncation search did not converge");
        }
    }
    return l;
}

// ---------------------------------------------------------------------------
// transfer function (Eq. TransferFn) and Algorithm BMTF
// ---------------------------------------------------------------------------
struct Transfer {
    int ell;
    double rhat[3];
    std::vector<cd> c;  // (i k / 4 pi) i^n (2n+1) h_n(k |r0|)
    Transfer(int ell_, double kappa, const double r0v[3]) : ell(ell_) {
        double r0 = std::sqrt(r0v[0] * r0v[0] + r0v[1] * r0v[1] + r0v[2] * r0v[2]);
        for (int k = 0; k < 3; ++k) rhat[k] = r0v[k] / r0;
        std::vector<cd> h;
        hankel_all(ell, kappa * r0, h);
        c.resize(ell + 1);
        const cd ipow[4] = {cd(1, 0), cd(0, 1), cd(-1, 0), cd(0, -1)};
        cd pre(0.0, kappa / (4.0 * kPi));
        for (int n = 0; n <= ell; ++n) c[n] = pre * ipow[n & 3] * (2.0 * n + 1.0) * h[n];
    }
    cd eval(double theta, double phi) const {
        double st = std::sin(theta);
        double s[3] = {std::cos(phi) * st, std::sin(phi) * st, std::cos(theta)};
        double t = s[0] * rhat[0] + s[1] * rhat[1] + s[2] * rhat[2];
        double p0 = 1.0, p1 = t;
        cd acc = c[0];
        if (ell >= 1) acc += c[1] * p1;
        for (int n = 1; n < ell; ++n) {
            double p2 = ((2.0 * n + 1.0) * t * p1 - n * p0) / (n + 1.0);
            acc += c[n + 1] * p2;
            p0 = p1;
            p1 = p2;
        }
        return acc;
    }
};

// theta-coefficients (freq -B..B, B = ntheta/2 - 1) of T^{s,L}(., phi) for one phi:
// sample 1/2 T on 2l+1 theta points, DFT, convolve with F[|sin|], truncate.
static void bmtf_coeffs(const Transfer& T, const Twiddle& tw, int ntheta, double phi,
                        std::vector<cd>& out) {
    const int ell = T.ell, m = 2 * ell + 1;
    std::vector<cd> samp(m), tf(m);
    for (int j = 0; j < m; ++j) samp[j] = 0.5 * T.eval(kTwoPi * j / m, phi);
    for (int f = -ell; f <= ell; ++f) {
        cd acc = 0.0;
        const int step = mod(f, m);          // (j * f) mod m, stepped with j
        int t = 0;
        for (int j = 0; j < m; ++j) {
            acc += samp[j] * tw.w[t];
            t += step;
            if (t >= m) t -= m;
        }
        tf[f + ell] = acc / (double)m;
    }
    const int b = ntheta / 2 - 1;
    // F[|sin|] at n - f for |n - f| <= b + ell; zero at odd arguments, so those terms are skipped
    std::vector<double> st(2 * (b + ell) + 1);
    for (int k = -(b + ell); k <= b + ell; ++k) st[k + b + ell] = s_tilde(k);
    out.assign(2 * b + 1, cd(0.0));
    for (int n = -b; n <= b; ++n) {
        cd acc = 0.0;
        const int f0 = ((n - (-ell)) % 2 == 0) ? -ell : -ell + 1;
        for (int f = f0; f <= ell; f += 2) acc += st[n - f + b + ell] * tf[f + ell];
        out[n + b] = acc;
    }
}

// sum_f coef_f exp(2 pi i f n_row / ntheta); twt = Twiddle(ntheta) (its inv() holds the same
// cos / sin values a direct evaluation of each angle gives)
static cd eval_theta(const std::vector<cd>& coef, const Twiddle& twt, int n_row) {
    const int b = twt.n / 2 - 1, n = twt.n;
    cd acc = 0.0;
    int t = mod(-(int64_t)b * n_row, n);   // (f * n_row) mod n, stepped with f
    for (int f = -b; f <= b; ++f) {
        acc += coef[f + b] * std::conj(twt.w[t]);
        t += n_row;
        if (t >= n) t -= n;
    }
    return acc;
}

// ---------------------------------------------------------------------------
// Algorithms Ntheta and Nphi
// ---------------------------------------------------------------------------
static int m_index(int nq, int n) {
    int a = std::abs(n);
    return (2 * a < nq) ? nq - a : a;
}

static int choose_ntheta(int ell, double kappa, double r, double r0, double eps_abs) {
    double r0v[3] = {0.0, 0.0, r0};
    Transfer T(ell, kappa, r0v);
    Twiddle tw(2 * ell + 1);
    int nmax = 2 * ell + 64;
    for (;;) {
        std::vector<cd> coef;
        bmtf_coeffs(T, tw, nmax, 0.0, coef);
        const int b = nmax / 2 - 1;
        std::vector<double> J(nmax + 1);
        bessel_jn_all(nmax, kappa * r, J.data());
        for (int nq = 2 * ell; nq <= nmax; nq += 2) {
            double s = 0.0;
            for (int f = -b; f <= b; ++f) s += std::abs(coef[f + b]) * std::fabs(J[m_index(nq, f)]);
            if (s < eps_abs / kFourPi2) return nq;
        }
        nmax *= 2;
    }
}

static std::vector<int> choose_nphi(int ell, double kappa, double r, double r0, int ntheta,
                                    double eps_abs) {
    double r0v[3] = {r0, 0.0, 0.0};
    Transfer T(ell, kappa, r0v);
    const int m = 2 * ell + 1;
    Twiddle tw(m);
    const int half = ntheta / 2;
    // T^{s,L}(theta_n, 2 pi p / m) for rows n <= half/2
    std::vector<std::vector<cd>> rows(half / 2 + 1, std::vector<cd>(m));
    const Twiddle twt(ntheta);
    // independent phi samples (each writes its own column)
#pragma omp parallel for schedule(dynamic, 4)
    for (int p = 0; p < m; ++p) {
        std::vector<cd> coef;
        bmtf_coeffs(T, tw, ntheta, kTwoPi * p / m, coef);
        for (int n = 0; n <= half / 2; ++n) rows[n][p] = eval_theta(coef, twt, n);
    }
    std::vector<int> nphi(half + 1, 0);
    // independent rows (each writes its own N_phi)
#pragma omp parallel for schedule(dynamic, 1)
    for (int n = 0; n <= half / 2; ++n) {
        std::vector<double> tt(m);
        for (int f = -ell; f <= ell; ++f) {
            cd acc = 0.0;
            for (int p = 0; p < m; ++p) acc += rows[n][p] * tw.fwd(p, f);
            tt[f + ell] = std::abs(acc / (double)m);
        }
        double x = kappa * r * std::sin(kTwoPi * n / ntheta);
        int nmax = 2 * ell + 64, found = 0;
        while (!found) {
            std::vector<double> J(nmax + 1);
            bessel_jn_all(nmax, x, J.data());
            for (int nq = 4; nq <= nmax; nq += 4) {
                double s = 0.0;
                for (int f = -ell; f <= ell; ++f) s += tt[f + ell] * std::fabs(J[m_index(nq, f)]);
                if (s < eps_abs / kFourPi2) {
                    found = nq;
                    break;
                }
            }
            nmax *= 2;
        }
        nphi[n] = found;
    }
    for (int n = 0; n <= half / 2; ++n) nphi[half - n] = nphi[n];
    return nphi;
}

static double round_off_estimate(int ell, double kappa, double r0, int64_t K, double u) {
    std::vector<cd> h;
    hankel_all(ell, kappa * r0, h);
    double s = 0.0;
    for (int n = 0; n <= ell; ++n) s += (2.0 * n + 1.0) * std::norm(h[n]);
    return u * kappa * r0 * std::sqrt(s) / std::sqrt((double)K);
}

static void plan_level(double kappa, double a, double eps_l, double alpha, int buffer, LevelPlan& lp) {
    lp.a = a;
    lp.alpha = alpha;
    lp.r = alpha * std::sqrt(3.0) * a;
    lp.r0 = (buffer + 1.0) * a;
    lp.eps_abs = eps_l / lp.r0;
    double d0 = -std::log10(eps_l);
    Quadrature& q = lp.quad;
    q.ell = choose_ell(kappa, lp.r, lp.r0, lp.eps_abs, d0);
    q.ntheta = (int)round_fft(choose_ntheta(q.ell, kappa, lp.r, lp.r0, lp.eps_abs), 2);
    // the device transforms work on lengths up to 1024; refuse before the O(l^3) N_phi search
    if (q.ntheta > 1024) throw std::runtime_error("N_theta above 1024 is not supported");
    std::vector<int> raw = choose_nphi(q.ell, kappa, lp.r, lp.r0, q.ntheta, lp.eps_abs);
    q.nphi.resize(raw.size());
    for (size_t n = 0; n < raw.size(); ++n) q.nphi[n] = (int)round_fft(raw[n], 4);
    q.finalize();
}

// ---------------------------------------------------------------------------
// T^{s,LL}: 34 canonical vectors by Algorithm BMTF + per-row anterpolation, 316 by reflection
// ---------------------------------------------------------------------------
// Per canonical vector: T^{s,L}(theta_n, phi_p) on the full phi grid (nfull samples, p <
// nfull/2 directly, the rest by Eq. NumSphereSym), then each row anterpolated nfull ->
// N_phi(theta_n).  The work is split into independent items (vector, phi sample) and
// (vector, row) so that all cores share one level's tables.
struct CanonWork {
    int d[3];
    Transfer T;
    std::vector<cd> grid;   // (half + 1) x nfull
    std::vector<cd> out;    // K
    CanonWork(const int dd[3], const LevelPlan& lp, double kappa)
        : d{dd[0], dd[1], dd[2]},
          T(lp.quad.ell, kappa, std::array<double, 3>{dd[0] * lp.a, dd[1] * lp.a, dd[2] * lp.a}.data()) {}
};

static void tsll_column(CanonWork& w, const LevelPlan& lp, const Twiddle& tw, const Twiddle& twt, int nfull, int p) {
    const int ntheta = lp.quad.ntheta, half = ntheta / 2;
    std::vector<cd> coef;
    bmtf_coeffs(w.T, tw, ntheta, kTwoPi * p / nfull, coef);
    for (int n = 0; n < ntheta; ++n) {
        cd v = eval_theta(coef, twt, n);
        if (n <= half) w.grid[(size_t)n * nfull + p] = v;
        int nn = (ntheta - n) % ntheta;  // f(theta_nn, phi_{p + nfull/2}) = f(theta_n, phi_p)
        if (nn <= half) w.grid[(size_t)nn * nfull + p + nfull / 2] = v;
    }
}

static void tsll_row(CanonWork& w, const LevelPlan& lp, const Twiddle& twf, int nfull, int n) {
    const Quadrature& q = lp.quad;
    const int np = q.nphi[n];
    const int b = std::min((nfull + 1) / 2, (np + 1) / 2) - 1;
    std::vector<cd> spec(2 * b + 1);
    for (int f = -b; f <= b; ++f) {
        cd acc = 0.0;
        const int step = mod(f, nfull);   // (p * f) mod nfull, stepped with p
        int t = 0;
        for (int p = 0; p < nfull; ++p) {
            acc += w.grid[(size_t)n * nfull + p] * twf.w[t];
            t += step;
            if (t >= nfull) t -= nfull;
        }
        spec[f + b] = acc / (double)nfull;
    }
    Twiddle twn(np);
    for (int j = 0; j < np; ++j) {
        cd acc = 0.0;
        int t = mod(-(int64_t)b * j, np);  // (j * f) mod np, stepped with f
        for (int f = -b; f <= b; ++f) {
            acc += spec[f + b] * std::conj(twn.w[t]);
            t += j;
            if (t >= np) t -= np;
        }
        w.out[(size_t)q.off[n] + j] = acc;
    }
}

// reflect the canonical table into vector d: T_d(s) = T_canon(P F s)
static std::vector<cd> reflect(const std::vector<cd>& canon, const Quadrature& q, const int d[3]) {
    const int half = q.ntheta / 2;
    const bool fx = d[0] < 0, fy = d[1] < 0, fz = d[2] < 0;
    const bool swap = std::abs(d[0]) < std::abs(d[1]);
    std::vector<cd> out((size_t)q.K);
    for (int n = 0; n <= half; ++n) {
        const int np = q.nphi[n];
        for (int m = 0; m < np; ++m) {
            int nn = n, mm = m;
            if (fx) mm = mod((int64_t)np / 2 - mm, np);
            if (fy) mm = mod(-(int64_t)mm, np);
            if (fz) nn = half - nn;
            if (swap) mm = mod((int64_t)np / 4 - mm, np);
            out[(size_t)q.off[n] + m] = canon[(size_t)q.off[nn] + mm];
        }
    }
    return out;
}

// canonical representative (x >= y >= 0, z >= 0) of an offset under the reflections
static std::array<int, 3> canonical(int di, int dj, int dk) {
    return {std::max(std::abs(di), std::abs(dj)), std::min(std::abs(di), std::abs(dj)), std::abs(dk)};
}

TableJob make_table_job(const LevelPlan& lp, double kappa, int buffer, const std::vector<char>& used) {
    const int D = transfer_span(buffer), W = transfer_width(buffer);
    TableJob job;
    job.ell = lp.quad.ell;
    job.nfull = 4 * ((2 * lp.quad.ell + 1 + 3) / 4);
    job.kappa = kappa;
    std::vector<std::array<int, 3>> canon;
    for (int di = -D; di <= D; ++di)
        for (int dj = -D; dj <= D; ++dj)
            for (int dk = -D; dk <= D; ++dk) {
                const int v = (di + D) * W * W + (dj + D) * W + (dk + D);
                if (!used[v]) continue;
                const std::array<int, 3> cv = canonical(di, dj, dk);
                if (std::find(canon.begin(), canon.end(), cv) == canon.end()) canon.push_back(cv);
            }
    std::sort(canon.begin(), canon.end());
    for (auto& cv : canon) {
        const double r0v[3] = {cv[0] * lp.a, cv[1] * lp.a, cv[2] * lp.a};
        Transfer T(lp.quad.ell, kappa, r0v);
        job.coef.insert(job.coef.end(), T.c.begin(), T.c.end());
        job.rhat.insert(job.rhat.end(), T.rhat, T.rhat + 3);
    }
    for (int di = -D; di <= D; ++di)
        for (int dj = -D; dj <= D; ++dj)
            for (int dk = -D; dk <= D; ++dk) {
                const int v = (di + D) * W * W + (dj + D) * W + (dk + D);
                if (!used[v]) continue;
                job.slot_canon.push_back(
                    (int32_t)(std::find(canon.begin(), canon.end(), canonical(di, dj, dk)) - canon.begin()));
                job.slot_flags.push_back((di < 0 ? 1 : 0) | (dj < 0 ? 2 : 0) | (dk < 0 ? 4 : 0) |
                                         (std::abs(di) < std::abs(dj) ? 8 : 0));
            }
    return job;
}

static void build_tables(LevelPlan& lp, double kappa, int buffer, const std::vector<char>& used) {
    const int D = transfer_span(buffer), W = transfer_width(buffer);
    lp.table.assign(transfer_slots(buffer), {});
    // canonical set: x >= y >= 0, z >= 0, max > buffer, restricted to what the lists use
    std::vector<std::array<int, 3>> canon;
    for (int di = -D; di <= D; ++di)
        for (int dj = -D; dj <= D; ++dj)
            for (int dk = -D; dk <= D; ++dk) {
                const int v = (di + D) * W * W + (dj + D) * W + (dk + D);
                if (!used[v]) continue;
                const std::array<int, 3> cv = canonical(di, dj, dk);
                if (std::find(canon.begin(), canon.end(), cv) == canon.end()) canon.push_back(cv);
            }
    std::sort(canon.begin(), canon.end());
    const Quadrature& q = lp.quad;
    const int ell = q.ell, half = q.ntheta / 2;
    const int nfull = 4 * ((2 * ell + 1 + 3) / 4);  // even, >= 2l+2: holds the phi band |m| <= l
    const Twiddle tw(2 * ell + 1), twt(q.ntheta), twf(nfull);
    std::vector<CanonWork> work;
    work.reserve(canon.size());
    for (auto& cv : canon) {
        work.emplace_back(cv.data(), lp, kappa);
        work.back().grid.assign((size_t)(half + 1) * nfull, cd(0.0));
        work.back().out.assign((size_t)q.K, cd(0.0));
    }
    const int nc = (int)canon.size(), ncol = nfull / 2, nrow = half + 1;
#pragma omp parallel for schedule(dynamic, 4)
    for (int it = 0; it < nc * ncol; ++it) tsll_column(work[it / ncol], lp, tw, twt, nfull, it % ncol);
#pragma omp parallel for schedule(dynamic, 2)
    for (int it = 0; it < nc * nrow; ++it) tsll_row(work[it / nrow], lp, twf, nfull, it % nrow);
    std::vector<std::vector<cd>> ct(canon.size());
    for (int c = 0; c < nc; ++c) ct[c] = std::move(work[c].out);
    for (int di = -D; di <= D; ++di)
        for (int dj = -D; dj <= D; ++dj)
            for (int dk = -D; dk <= D; ++dk) {
                const int v = (di + D) * W * W + (dj + D) * W + (dk + D);
                if (!used[v]) continue;
                int d[3] = {di, dj, dk};
                size_t c = std::find(canon.begin(), canon.end(), canonical(di, dj, dk)) - canon.begin();
                lp.table[v] = reflect(ct[c], lp.quad, d);
            }
}

// ---------------------------------------------------------------------------
// tree
// ---------------------------------------------------------------------------
static uint64_t morton(uint32_t ix, uint32_t iy, uint32_t iz, int depth) {
    uint64_t k = 0;
    for (int b = 0; b < depth; ++b) {
        k |= (uint64_t)((ix >> b) & 1u) << (3 * b + 2);
        k |= (uint64_t)((iy >> b) & 1u) << (3 * b + 1);
        k |= (uint64_t)((iz >> b) & 1u) << (3 * b);
    }
    return k;
}

static void demorton(uint64_t k, int depth, int32_t out[3]) {
    out[0] = out[1] = out[2] = 0;
    for (int b = 0; b < depth; ++b) {
        out[0] |= (int32_t)((k >> (3 * b + 2)) & 1u) << b;
        out[1] |= (int32_t)((k >> (3 * b + 1)) & 1u) << b;
        out[2] |= (int32_t)((k >> (3 * b)) & 1u) << b;
    }
}

// ascending sort on all threads (the values sorted here are plain integers, so the result is
// the same as a serial sort)
static void psort(std::vector<uint64_t>& v) { __gnu_parallel::sort(v.begin(), v.end()); }

// keys at depth kTreeBits
static void leaf_keys(const std::vector<double>& p, int64_t n, const double corner[3], double side,
                      std::vector<uint64_t>& key) {
    const double nb = (double)(1u << kTreeBits);
    const double scale = nb / side;
    key.resize(n);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        uint32_t c[3];
        for (int k = 0; k < 3; ++k) {
            double v = std::floor((p[3 * i + k] - corner[k]) * scale);
            if (v < 0.0) v = 0.0;
            if (v > nb - 1.0) v = nb - 1.0;
            c[k] = (uint32_t)v;
        }
        key[i] = morton(c[0], c[1], c[2], kTreeBits);
    }
}

static int max_run(const std::vector<uint64_t>& sorted_keys, int shift) {
    int best = 0, run = 0;
    for (size_t i = 0; i < sorted_keys.size(); ++i) {
        uint64_t k = sorted_keys[i] >> shift;
        run = (i > 0 && (sorted_keys[i - 1] >> shift) == k) ? run + 1 : 1;
        best = std::max(best, run);
    }
    return best;
}

static int64_t find_key(const std::vector<uint64_t>& keys, uint64_t k) {
    auto it = std::lower_bound(keys.begin(), keys.end(), k);
    if (it == keys.end() || *it != k) return -1;
    return it - keys.begin();
}

static void build_tree(HostPlan& hp) {
    // sources and targets the same point set: one key array and one sort serve both
    const bool same = hp.ns == hp.nt && hp.src == hp.tgt;
    std::vector<uint64_t> ks, kt;
    leaf_keys(hp.src, hp.ns, hp.corner, hp.side, ks);
    if (!same) leaf_keys(hp.tgt, hp.nt, hp.corner, hp.side, kt);
    const std::vector<uint64_t>& ktr = same ? ks : kt;
    const int D = hp.lf;
    const int shift = 3 * (kTreeBits - D);
    // sort by depth-D key, ties by original index: one sort of packed (key, index) words when
    // both fit in 64 bits (3 D key bits + index bits), else a stable index sort
    auto sort_perm = [&](const std::vector<uint64_t>& k, std::vector<int64_t>& perm) {
        const int64_t n = (int64_t)k.size();
        perm.resize(n);
        int ibits = 1;
        while (ibits < 63 && (int64_t(1) << ibits) < n) ++ibits;
        if (3 * D + ibits <= 64) {
            std::vector<uint64_t> w(n);
            for (int64_t i = 0; i < n; ++i) w[i] = ((k[i] >> shift) << ibits) | (uint64_t)i;
            psort(w);   // the words are distinct: the order is unique
            const uint64_t mask = (ibits == 64) ? ~uint64_t(0) : ((uint64_t(1) << ibits) - 1);
            for (int64_t i = 0; i < n; ++i) perm[i] = (int64_t)(w[i] & mask);
        } else {
            std::iota(perm.begin(), perm.end(), 0);
            std::stable_sort(perm.begin(), perm.end(),
                             [&](int64_t a, int64_t b) { return (k[a] >> shift) < (k[b] >> shift); });
        }
    };
    sort_perm(ks, hp.src_perm);
    if (same) hp.tgt_perm = hp.src_perm;
    else sort_perm(kt, hp.tgt_perm);
    std::vector<uint64_t> allk;
    allk.reserve(ks.size() + (same ? 0 : kt.size()));
    for (auto k : ks) allk.push_back(k >> shift);
    if (!same)
        for (auto k : kt) allk.push_back(k >> shift);
    psort(allk);
    allk.erase(std::unique(allk.begin(), allk.end()), allk.end());
    hp.levels.assign(D + 1, TreeLevel());
    // adaptive trees: depth-D keys of the points in tree order, and level-l keys of the sorted
    // points (for the per-box subtree ranges)
    std::vector<uint64_t> lks, lkt, sds, sdt;
    if (hp.adaptive) {
        auto sorted_keys = [&](const std::vector<uint64_t>& k, const std::vector<int64_t>& perm, std::vector<uint64_t>& out) {
            out.resize(perm.size());
#pragma omp parallel for schedule(static)
            for (int64_t p = 0; p < (int64_t)perm.size(); ++p) out[p] = k[perm[p]] >> shift;
        };
        sorted_keys(ks, hp.src_perm, sds);
        if (!same) sorted_keys(ktr, hp.tgt_perm, sdt);
    }
    for (int l = 0; l <= D; ++l) {
        TreeLevel& L = hp.levels[l];
        for (auto k : allk) {
            uint64_t kl = k >> (3 * (D - l));
            if (!L.key.empty() && L.key.back() == kl) continue;
            if (hp.adaptive && l > 0) {
                // boxes exist only below split boxes
                const TreeLevel& U = hp.levels[l - 1];
                const int64_t pb = find_key(U.key, kl >> 3);
                if (pb < 0 || !U.split[pb]) continue;
            }
            L.key.push_back(kl);
        }
        const int64_t nb = L.nbox();
        L.idx.resize(3 * nb);
        L.center.resize(3 * nb);
        L.parent.assign(nb, -1);
        const double h = hp.side / (double)(1u << l);
        for (int64_t b = 0; b < nb; ++b) {
            demorton(L.key[b], l, &L.idx[3 * b]);
            for (int k = 0; k < 3; ++k)
                L.center[3 * b + k] = hp.corner[k] + ((double)L.idx[3 * b + k] + 0.5) * h;
            if (l > 0) L.parent[b] = (int32_t)find_key(hp.levels[l - 1].key, L.key[b] >> 3);
        }
        if (l > 0) {
            TreeLevel& P = hp.levels[l - 1];
            P.child_start.assign(P.nbox(), 0);
            P.child_count.assign(P.nbox(), 0);
            for (int64_t b = nb - 1; b >= 0; --b) {
                P.child_start[L.parent[b]] = (int32_t)b;
                P.child_count[L.parent[b]]++;
            }
        }
        if (hp.adaptive) {
            // subtree ranges: the sorted points whose level-l key is the box's key
            auto sub = [&](const std::vector<uint64_t>& sorted_d, std::vector<uint64_t>& lk,
                           std::vector<int32_t>& start, std::vector<int32_t>& count) {
                lk.resize(sorted_d.size());
#pragma omp parallel for schedule(static)
                for (int64_t p = 0; p < (int64_t)sorted_d.size(); ++p) lk[p] = sorted_d[p] >> (3 * (D - l));
                start.resize(nb);
                count.resize(nb);
                for (int64_t b = 0; b < nb; ++b) {
                    auto lo = std::lower_bound(lk.begin(), lk.end(), L.key[b]);
                    auto hi = std::upper_bound(lo, lk.end(), L.key[b]);
                    start[b] = (int32_t)(lo - lk.begin());
                    count[b] = (int32_t)(hi - lo);
                }
            };
            sub(sds, lks, L.s_start, L.s_count);
            if (same) {
                lkt = lks;
                L.t_start = L.s_start;
                L.t_count = L.s_count;
            } else {
                sub(sdt, lkt, L.t_start, L.t_count);
            }
            // split: above level 2, more than max_leaf sources or targets, or crowded (the
            // other level-l cubes within Chebyshev distance buffer hold more than
            // (2 buffer + 1)^3 max_leaf sources or targets)
            const int bw = hp.buffer, n1 = 1 << l;
            const int64_t lim = (int64_t)(2 * bw + 1) * (2 * bw + 1) * (2 * bw + 1) * hp.max_leaf;
            L.split.assign(nb, 0);
#pragma omp parallel for schedule(static)
            for (int64_t b = 0; b < nb; ++b) {
                bool sp = l < 2 || L.s_count[b] > hp.max_leaf || L.t_count[b] > hp.max_leaf;
                if (!sp && l < D && L.s_count[b] + L.t_count[b] > 0) {
                    const int32_t* ib = &L.idx[3 * b];
                    int64_t cs = 0, ct = 0;
                    for (int dx = -bw; dx <= bw; ++dx)
                        for (int dy = -bw; dy <= bw; ++dy)
                            for (int dz = -bw; dz <= bw; ++dz) {
                                const int c[3] = {ib[0] + dx, ib[1] + dy, ib[2] + dz};
                                if ((dx | dy | dz) == 0 || c[0] < 0 || c[1] < 0 || c[2] < 0 || c[0] >= n1 ||
                                    c[1] >= n1 || c[2] >= n1)
                                    continue;
                                const uint64_t k = morton(c[0], c[1], c[2], l);
                                cs += std::upper_bound(lks.begin(), lks.end(), k) - std::lower_bound(lks.begin(), lks.end(), k);
                                ct += std::upper_bound(lkt.begin(), lkt.end(), k) - std::lower_bound(lkt.begin(), lkt.end(), k);
                            }
                    sp = cs > lim || ct > lim;
                }
                L.split[b] = l < D && sp;
            }
        } else {
            L.split.assign(nb, l < D ? 1 : 0);
        }
        for (int64_t b = 0; b < nb; ++b)
            if (!L.split[b]) L.leaf_pos.push_back((int32_t)b);
    }
    // leaf point ranges
    TreeLevel& leaf = hp.levels[D];
    const int64_t nb = leaf.nbox();
    auto ranges = [&](const std::vector<uint64_t>& k, const std::vector<int64_t>& perm,
                      std::vector<int32_t>& start, std::vector<int32_t>& count) {
        start.assign(nb, 0);
        count.assign(nb, 0);
        int64_t b = 0;
        for (int64_t p = 0; p < (int64_t)perm.size(); ++p) {
            uint64_t kk = k[perm[p]] >> shift;
            while (leaf.key[b] < kk) ++b;
            if (count[b] == 0) start[b] = (int32_t)p;
            count[b]++;
        }
        for (int64_t i = 0; i < nb; ++i)
            if (count[i] == 0) start[i] = (i > 0) ? start[i - 1] + count[i - 1] : 0;
    };
    if (hp.adaptive) {
        // leaves of all levels in Morton order of their first depth-D key
        std::vector<std::array<int64_t, 3>> lv;
        for (int l = 0; l <= D; ++l)
            for (int32_t b : hp.levels[l].leaf_pos)
                lv.push_back({(int64_t)(hp.levels[l].key[b] << (3 * (D - l))), l, b});
        std::sort(lv.begin(), lv.end());
        const int64_t nl = (int64_t)lv.size();
        hp.leaf_level.resize(nl);
        hp.leaf_box.resize(nl);
        hp.src_start.resize(nl);
        hp.src_count.resize(nl);
        hp.tgt_start.resize(nl);
        hp.tgt_count.resize(nl);
        std::vector<uint64_t> first(nl);
        for (int64_t g = 0; g < nl; ++g) {
            const TreeLevel& L = hp.levels[lv[g][1]];
            const int32_t b = (int32_t)lv[g][2];
            first[g] = (uint64_t)lv[g][0];
            hp.leaf_level[g] = (int32_t)lv[g][1];
            hp.leaf_box[g] = b;
            hp.src_start[g] = L.s_start[b];
            hp.src_count[g] = L.s_count[b];
            hp.tgt_start[g] = L.t_start[b];
            hp.tgt_count[g] = L.t_count[b];
        }
        // near lists: leaves C whose ancestor at level m = min(l_B, l_C) neighbours leaf B's
        // ancestor there: (i) every leaf under a level-l_B neighbour of B (l_C >= l_B);
        // (ii) leaves of a coarser level m that neighbour B's level-m ancestor
        const int bw = hp.buffer;
        std::vector<std::vector<int32_t>> nf(nl);
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t g = 0; g < nl; ++g) {
            const int lb = hp.leaf_level[g];
            const int32_t* ib = &hp.levels[lb].idx[3 * hp.leaf_box[g]];
            for (int m = 0; m <= lb; ++m) {
                const TreeLevel& M = hp.levels[m];
                const int n1 = 1 << m;
                const int32_t a[3] = {ib[0] >> (lb - m), ib[1] >> (lb - m), ib[2] >> (lb - m)};
                for (int dx = -bw; dx <= bw; ++dx)
                    for (int dy = -bw; dy <= bw; ++dy)
                        for (int dz = -bw; dz <= bw; ++dz) {
                            const int c[3] = {a[0] + dx, a[1] + dy, a[2] + dz};
                            if (c[0] < 0 || c[1] < 0 || c[2] < 0 || c[0] >= n1 || c[1] >= n1 || c[2] >= n1) continue;
                            const int64_t nbx = find_key(M.key, morton(c[0], c[1], c[2], m));
                            if (nbx < 0) continue;
                            const uint64_t k0 = M.key[nbx] << (3 * (D - m));
                            if (m == lb) {
                                const uint64_t k1 = (M.key[nbx] + 1) << (3 * (D - m));
                                auto lo = std::lower_bound(first.begin(), first.end(), k0);
                                auto hi = std::lower_bound(lo, first.end(), k1);
                                for (auto it = lo; it != hi; ++it) nf[g].push_back((int32_t)(it - first.begin()));
                            } else if (!M.split[nbx]) {
                                nf[g].push_back((int32_t)(std::lower_bound(first.begin(), first.end(), k0) - first.begin()));
                            }
                        }
            }
            std::sort(nf[g].begin(), nf[g].end());
        }
        hp.noff.assign(nl + 1, 0);
        for (int64_t g = 0; g < nl; ++g) hp.noff[g + 1] = hp.noff[g] + (int32_t)nf[g].size();
        hp.nidx.resize(hp.noff.back());
        hp.p2p_pairs = 0;
        hp.p2p_self_pairs = 0;
        for (int64_t g = 0; g < nl; ++g) {
            for (size_t t = 0; t < nf[g].size(); ++t) {
                hp.nidx[hp.noff[g] + t] = nf[g][t];
                hp.p2p_pairs += (int64_t)hp.tgt_count[g] * hp.src_count[nf[g][t]];
            }
            hp.p2p_self_pairs += (int64_t)hp.tgt_count[g] * hp.src_count[g];
        }
    } else {
        ranges(ks, hp.src_perm, hp.src_start, hp.src_count);
        ranges(ktr, hp.tgt_perm, hp.tgt_start, hp.tgt_count);
        hp.leaf_level.assign(nb, D);
        hp.leaf_box.resize(nb);
        std::iota(hp.leaf_box.begin(), hp.leaf_box.end(), 0);
    }
    // interaction lists: children of the parent's neighbours (Chebyshev distance <= buffer)
    // that are not neighbours of the box itself
    const int bw = hp.buffer, TD = transfer_span(bw), TW = transfer_width(bw);
    for (int l = 2; l <= D; ++l) {
        TreeLevel& L = hp.levels[l];
        const int n1 = 1 << l;
        L.ioff.assign(L.nbox() + 1, 0);
        std::vector<std::vector<std::array<int64_t, 3>>> found(L.nbox());
#pragma omp parallel for schedule(static)
        for (int64_t a = 0; a < L.nbox(); ++a) {
            const int32_t* ia = &L.idx[3 * a];
            for (int px = -bw; px <= bw; ++px)
                for (int py = -bw; py <= bw; ++py)
                    for (int pz = -bw; pz <= bw; ++pz)
                        for (int c = 0; c < 8; ++c) {
                            int ib[3] = {((ia[0] >> 1) + px) * 2 + ((c >> 2) & 1),
                                         ((ia[1] >> 1) + py) * 2 + ((c >> 1) & 1),
                                         ((ia[2] >> 1) + pz) * 2 + (c & 1)};
                            bool ok = true;
                            int dmax = 0;
                            for (int k = 0; k < 3; ++k) {
                                if (ib[k] < 0 || ib[k] >= n1) ok = false;
                                dmax = std::max(dmax, std::abs(ib[k] - ia[k]));
                            }
                            if (!ok || dmax <= bw) continue;
                            int64_t b = find_key(L.key, morton(ib[0], ib[1], ib[2], l));
                            if (b < 0) continue;
                            int v = (ib[0] - ia[0] + TD) * TW * TW + (ib[1] - ia[1] + TD) * TW + (ib[2] - ia[2] + TD);
                            found[a].push_back({(int64_t)L.key[b], b, v});
                        }
            std::sort(found[a].begin(), found[a].end());
        }
        for (int64_t a = 0; a < L.nbox(); ++a) L.ioff[a + 1] = L.ioff[a] + (int32_t)found[a].size();
        L.iidx.resize(L.ioff.back());
        L.iv.resize(L.ioff.back());
        for (int64_t a = 0; a < L.nbox(); ++a)
            for (size_t t = 0; t < found[a].size(); ++t) {
                L.iidx[L.ioff[a] + t] = (int32_t)found[a][t][1];
                L.iv[L.ioff[a] + t] = (int32_t)found[a][t][2];
            }
    }
    if (hp.adaptive) return;
    // neighbour lists at the leaf level
    hp.noff.assign(nb + 1, 0);
    std::vector<std::vector<std::pair<uint64_t, int64_t>>> nf(nb);
    const int n1 = 1 << D;
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < nb; ++a) {
        const int32_t* ia = &leaf.idx[3 * a];
        for (int dx = -bw; dx <= bw; ++dx)
            for (int dy = -bw; dy <= bw; ++dy)
                for (int dz = -bw; dz <= bw; ++dz) {
                    int ib[3] = {ia[0] + dx, ia[1] + dy, ia[2] + dz};
                    if (ib[0] < 0 || ib[1] < 0 || ib[2] < 0 || ib[0] >= n1 || ib[1] >= n1 || ib[2] >= n1)
                        continue;
                    int64_t b = find_key(leaf.key, morton(ib[0], ib[1], ib[2], D));
                    if (b >= 0) nf[a].push_back({leaf.key[b], b});
                }
        std::sort(nf[a].begin(), nf[a].end());
    }
    for (int64_t a = 0; a < nb; ++a) hp.noff[a + 1] = hp.noff[a] + (int32_t)nf[a].size();
    hp.nidx.resize(hp.noff.back());
    hp.p2p_pairs = 0;
    for (int64_t a = 0; a < nb; ++a)
        for (size_t t = 0; t < nf[a].size(); ++t) {
            hp.nidx[hp.noff[a] + t] = (int32_t)nf[a][t].second;
            hp.p2p_pairs += (int64_t)hp.tgt_count[a] * hp.src_count[nf[a][t].second];
        }
    hp.p2p_self_pairs = 0;
    for (int64_t a = 0; a < nb; ++a) hp.p2p_self_pairs += (int64_t)hp.tgt_count[a] * hp.src_count[a];
}

// ---------------------------------------------------------------------------
// active levels for one buffer choice: alpha ladder outer, precision inner, precision never
// decreasing with depth; *lf = the deepest accepted level (levels stop at the first failure)
static std::vector<LevelPlan> plan_levels(const HostPlan& hp, int buffer, int dmax, int* lf_out) {
    std::vector<LevelPlan> lps(kMaxLevels);
    std::vector<int> allowed = (hp.precision == 1) ? std::vector<int>{kFP32, kDF, kFP64}
                                                   : std::vector<int>{kFP64};
    int lf = 1;
    for (int l = 2; l <= dmax && l < kMaxLevels; ++l) {
        // one buffer box: only boxes of about a wavelength or larger use the diagonal form
        if (hp.kappa * (hp.side / (double)(1u << l)) < min_ka(buffer)) break;
        bool ok = false;
        for (double alpha : hp.alphas) {
            LevelPlan cand;
            plan_level(hp.kappa, hp.side / (double)(1u << l), hp.eps_l, alpha, buffer, cand);
            for (int p : allowed) {
                const double u = std::ldexp(1.0, p == kFP32 ? -24 : (p == kDF ? -48 : -53));
                const double f = (p == kFP32) ? 1.0 : 1.0 / 16.0;
                double est = round_off_estimate(cand.quad.ell, hp.kappa, cand.r0, cand.quad.K, u);
                if (est <= hp.eps_l * f) {
                    cand.prec = p;
                    cand.est = est;
                    lps[l] = cand;
                    ok = true;
                    allowed.erase(allowed.begin(), std::find(allowed.begin(), allowed.end(), p));
                    break;
                }
            }
            if (ok) break;
        }
        if (!ok) break;
        lf = l;
    }
    if (dmax < 2) lf = dmax;
    *lf_out = lf;
    return lps;
}

// ---------------------------------------------------------------------------
// Plan-shape tuner: the number of buffer boxes (1 or 2, Section 3.3.3) and the leaf level
// L_f <= the deepest stable level, chosen by a cost model of one apply.  Two buffer boxes
// shrink l and keep deeper levels stable (smaller near field, cheaper leaf precision) but
// lengthen interaction lists (up to 875 entries) and neighbour lists (5^3 boxes); a shallower
// leaf trades far-field work for near-field pairs.  The model counts, for each candidate,
// near-field pairs, (point, antipodal sample pair) products of S2M and L2T, interaction-list
// entries x samples of M2L and boxes x samples of the re-quadratures, and weighs them with
// per-unit times measured on a GB300 (stage times of the benchmark workloads).
// ---------------------------------------------------------------------------
namespace {

// seconds per unit on a GB300 (2070 MHz); R = right-hand sides
struct UnitCost {
    double near_f32_sym = 1.32e-12, near_f32_boxpair = 0.65e-9;  // symmetric float32, R = 1: per
                                                                 // ordered pair, ordered box pair
    double near_f32 = 2.7e-12;        // per pair and group of four RHS (one-way float32)
    double near_tc = 0.27e-12;        // per pair and RHS (mma.sync tensor-core form, 8 <= R < 16)
    double near_tc5 = 8.0e-9;         // per (128-target chunk, 16-source tile, 64-RHS pass), tcgen05 form
    double near_df = 7.3e-12;         // per pair and group of four RHS
    double near_f64 = 1.0e-10;        // per pair and RHS
    double pw_f32 = 1.5e-12, pw_f32_rhs = 0.42e-12;  // per (point, antipodal pair): per plane
                                                      // wave (one per 1, 4 or 16 RHS) + per RHS
    double pw_df = 2.9e-12, pw_df_rhs = 3.15e-12;
    double pw_f64_tab = 6.5e-12;      // per (point, pair, RHS), float64 tables
    double pw_f64 = 67e-12, pw_f64_rhs = 6.5e-12;
    double m2l_f32 = 1.28e-12, m2l_df = 2.5e-12, m2l_f64 = 11e-12;   // per (entry, sample, RHS)
    double requad = 1.1e-10;          // per (box, sample, RHS) of M2M and again of L2L
};

struct LevelCounts {
    std::vector<uint64_t> key;     // nonempty boxes, ascending
    std::vector<int64_t> ns, nt;   // sources / targets per box
};

// boxes of one level with their point counts, from sorted depth-20 keys
LevelCounts level_counts(const std::vector<uint64_t>& ks, const std::vector<uint64_t>& kt, int l) {
    LevelCounts c;
    const int sh = 3 * (kTreeBits - l);
    size_t i = 0, j = 0;
    while (i < ks.size() || j < kt.size()) {
        const uint64_t a = i < ks.size() ? ks[i] >> sh : ~uint64_t(0);
        const uint64_t b = j < kt.size() ? kt[j] >> sh : ~uint64_t(0);
        const uint64_t k = std::min(a, b);
        int64_t ns = 0, nt = 0;
        while (i < ks.size() && (ks[i] >> sh) == k) ++i, ++ns;
        while (j < kt.size() && (kt[j] >> sh) == k) ++j, ++nt;
        c.key.push_back(k);
        c.ns.push_back(ns);
        c.nt.push_back(nt);
    }
    return c;
}

// sum over boxes of f(box, neighbour) for neighbours within Chebyshev distance bw
template <typename F>
void for_neighbours(const std::vector<uint64_t>& keys, int l, int bw, F f) {
    const int n1 = 1 << l;
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < (int64_t)keys.size(); ++a) {
        int32_t ia[3];
        demorton(keys[a], l, ia);
        for (int dx = -bw; dx <= bw; ++dx)
            for (int dy = -bw; dy <= bw; ++dy)
                for (int dz = -bw; dz <= bw; ++dz) {
                    const int ib[3] = {ia[0] + dx, ia[1] + dy, ia[2] + dz};
                    if (ib[0] < 0 || ib[1] < 0 || ib[2] < 0 || ib[0] >= n1 || ib[1] >= n1 || ib[2] >= n1) continue;
                    const int64_t b = find_key(keys, morton(ib[0], ib[1], ib[2], l));
                    if (b >= 0) f(a, b);
                }
    }
}

}  // namespace

// Predicted apply time (s) of the adaptive tree with b buffer boxes and leaf level L: the tree,
// its near lists and interaction lists are built as for the apply; near-field pairs, leaf
// plane-wave products per leaf level, list entries and re-quadrature samples are weighed as in
// the uniform model (no float64 leaf tables: adaptive plans do not build them).
static double adaptive_cost(const HostPlan& hp, const std::vector<LevelPlan>& lps, int b, int L, const UnitCost& uc,
                            HostPlan& t) {
    t = HostPlan();
    t.src = hp.src;
    t.tgt = hp.tgt;
    t.ns = hp.ns;
    t.nt = hp.nt;
    t.max_leaf = hp.max_leaf;
    t.adaptive = 1;
    t.buffer = b;
    t.lf = L;
    for (int k = 0; k < 3; ++k) t.corner[k] = hp.corner[k];
    t.side = hp.side;
    build_tree(t);
    const double R = hp.model_rhs;
    const double g4 = std::ceil(R / 4.0);
    double pairs = 0.0, unit_tiles = 0.0;
    const double boxpairs = (double)t.nidx.size();
    for (size_t g = 0; g < t.leaf_level.size(); ++g) {
        double tl = 0.0;
        for (int32_t k = t.noff[g]; k < t.noff[g + 1]; ++k) {
            pairs += (double)t.tgt_count[g] * (double)t.src_count[t.nidx[k]];
            tl += (double)((t.src_count[t.nidx[k]] + 15) / 16);
        }
        unit_tiles += (double)((t.tgt_count[g] + 127) / 128) * tl;
    }
    double c = 0.0;
    if (hp.model_near == kFP32) {
        if (hp.model_sym && R == 1) c += pairs * uc.near_f32_sym + boxpairs * uc.near_f32_boxpair;
        else if (R >= 16) c += unit_tiles * std::ceil(R / 64.0) * uc.near_tc5;
        else if (R >= 8) c += pairs * R * uc.near_tc;
        else c += pairs * g4 * uc.near_f32;
    } else if (hp.model_near == kDF) {
        c += pairs * g4 * uc.near_df;
    } else {
        c += pairs * R * uc.near_f64;
    }
    for (int l = 2; l <= L; ++l) {
        const LevelPlan& lp = lps[l];
        const TreeLevel& T = t.levels[l];
        // S2M and L2T of this level's leaves
        double pts = 0.0;
        for (int32_t bx : T.leaf_pos) pts += (double)T.s_count[bx] + (double)T.t_count[bx];
        const double npair = (double)lp.quad.K / 2.0;
        if (lp.prec == kFP32) {
            const double rc = R >= 16 ? 16.0 : (R > 1 ? 4.0 : 1.0);
            c += pts * npair * (std::ceil(R / rc) * uc.pw_f32 + R * uc.pw_f32_rhs);
        } else if (lp.prec == kDF) {
            c += pts * npair * (uc.pw_df + R * uc.pw_df_rhs);
        } else {
            c += pts * npair * (uc.pw_f64 + R * uc.pw_f64_rhs);
        }
        const double cm = lp.prec == kFP32 ? uc.m2l_f32 : (lp.prec == kDF ? uc.m2l_df : uc.m2l_f64);
        c += (double)T.iidx.size() * (double)lp.quad.K * R * cm;
        if (l >= 3) c += 2.0 * uc.requad * R * (double)T.nbox() * (double)lp.quad.K;
    }
    return c;
}

// ks, kt: depth-kTreeBits keys of the sources and targets, ascending
static void tune_plan_shape(HostPlan& hp, const std::vector<uint64_t>& ks, const std::vector<uint64_t>& kt) {
    const UnitCost uc;
    const double R = hp.model_rhs;
    std::vector<LevelPlan> lps[3];
    int lfb[3] = {1, 1, 1};
    for (int b = 1; b <= 2; ++b) lps[b] = plan_levels(hp, b, hp.occ_depth, &lfb[b]);
    const int lmax = std::max(lfb[1], lfb[2]);
    std::vector<LevelCounts> lc(lmax + 1);
    for (int l = 1; l <= lmax; ++l) lc[l] = level_counts(ks, kt, l);
    double best = -1.0;
    int bb = 1, bl = lfb[1];
    for (int b = 1; b <= 2; ++b) {
        if (lfb[b] < 2) continue;
        // interaction-list lengths: children of the parent's neighbours minus own neighbours
        std::vector<double> ilist(lfb[b] + 1, 0.0);
        for (int l = 2; l <= lfb[b]; ++l) {
            const LevelCounts& P = lc[l - 1];
            const LevelCounts& C = lc[l];
            std::vector<int64_t> nchild(P.key.size(), 0), cand(P.key.size(), 0), own(C.key.size(), 0);
            for (uint64_t k : C.key) nchild[find_key(P.key, k >> 3)]++;
            for_neighbours(P.key, l - 1, b, [&](int64_t a, int64_t n) { cand[a] += nchild[n]; });
            for_neighbours(C.key, l, b, [&](int64_t a, int64_t) { own[a]++; });
            double tot = 0.0;
            for (size_t a = 0; a < C.key.size(); ++a) tot += (double)(cand[find_key(P.key, C.key[a] >> 3)] - own[a]);
            ilist[l] = tot;
        }
        for (int L = 2; L <= lfb[b]; ++L) {
            // near field at leaf level L
            const LevelCounts& F = lc[L];
            std::vector<double> pr(F.key.size(), 0.0), bpr(F.key.size(), 0.0), tl(F.key.size(), 0.0);
            for_neighbours(F.key, L, b, [&](int64_t a, int64_t n) {
                pr[a] += (double)F.nt[a] * (double)F.ns[n];
                bpr[a] += 1.0;
                tl[a] += (double)((F.ns[n] + 15) / 16);
            });
            double pairs = 0.0, boxpairs = 0.0, unit_tiles = 0.0;
            for (size_t a = 0; a < F.key.size(); ++a) {
                pairs += pr[a];
                boxpairs += bpr[a];
                unit_tiles += (double)((F.nt[a] + 127) / 128) * tl[a];
            }
            double t = 0.0;
            const double g4 = std::ceil(R / 4.0);
            if (hp.model_near == kFP32) {
                if (hp.model_sym && R == 1) t += pairs * uc.near_f32_sym + boxpairs * uc.near_f32_boxpair;
                else if (R >= 16) t += unit_tiles * std::ceil(R / 64.0) * uc.near_tc5;
                else if (R >= 8) t += pairs * R * uc.near_tc;
                else t += pairs * g4 * uc.near_f32;
            } else if (hp.model_near == kDF) {
                t += pairs * g4 * uc.near_df;
            } else {
                t += pairs * R * uc.near_f64;
            }
            // S2M and L2T at the leaf
            const LevelPlan& leaf = lps[b][L];
            const double npair = (double)leaf.quad.K / 2.0, pts = (double)(hp.ns + hp.nt);
            if (leaf.prec == kFP32) {
                const double rc = R >= 16 ? 16.0 : (R > 1 ? 4.0 : 1.0);   // RHS per plane wave
                t += pts * npair * (std::ceil(R / rc) * uc.pw_f32 + R * uc.pw_f32_rhs);
            } else if (leaf.prec == kDF) {
                t += pts * npair * (uc.pw_df + R * uc.pw_df_rhs);
            } else {
                const double bytes = npair * 16.0 * (double)(hp.ns + (hp.model_sym ? 0 : hp.nt));
                const double cap = hp.model_table_bytes > 0 ? (double)hp.model_table_bytes : 96.0 * 1073741824.0;
                if (hp.model_table_bytes != 0 && bytes <= cap) t += pts * npair * R * uc.pw_f64_tab;
                else t += pts * npair * (uc.pw_f64 + R * uc.pw_f64_rhs);
            }
            // M2L and the re-quadratures of levels 2..L
            for (int l = 2; l <= L; ++l) {
                const LevelPlan& lp = lps[b][l];
                const double c = lp.prec == kFP32 ? uc.m2l_f32 : (lp.prec == kDF ? uc.m2l_df : uc.m2l_f64);
                t += ilist[l] * (double)lp.quad.K * R * c;
                if (l >= 3) t += 2.0 * uc.requad * R * (double)lc[l].key.size() * (double)lp.quad.K;
            }
            hp.predicted_ms[b][L] = 1e3 * t;
            if (best < 0.0 || t < best) {
                best = t;
                bb = b;
                bl = L;
            }
        }
    }
    if (hp.adaptive) {
        // adaptive trees: the uniform counts above overstate the far field of sparse regions
        // and understate the leaf levels; cost the adaptive tree itself (built as the apply
        // would use it, with the same per-unit times) at the uniform choice of each buffer
        // whose uniform prediction is within 2.5x of the best and one level deeper (sparse
        // regions stop early, so deeper leaves cost less than in a uniform tree), choose among
        // those, and keep the chosen candidate's tree for the plan (each candidate costs one
        // tree build)
        int best_l[3] = {0, 0, 0};
        double best_t[3] = {-1.0, -1.0, -1.0};
        for (int b = 1; b <= 2; ++b)
            for (int L = 2; L <= lfb[b]; ++L)
                if (hp.predicted_ms[b][L] > 0.0 && (best_t[b] < 0.0 || hp.predicted_ms[b][L] < best_t[b])) {
                    best_t[b] = hp.predicted_ms[b][L];
                    best_l[b] = L;
                }
        const double uni = 1e3 * best;
        for (int b = 1; b <= 2; ++b)
            for (int L = 0; L < kMaxLevels; ++L) hp.predicted_ms[b][L] = 0.0;
        best = -1.0;
        for (int b = 1; b <= 2; ++b) {
            if (lfb[b] < 2 || best_t[b] < 0.0 || best_t[b] > 2.5 * uni) continue;
            for (int L = best_l[b]; L <= std::min(lfb[b], best_l[b] + 1); ++L) {
                HostPlan cand;
                const double t = adaptive_cost(hp, lps[b], b, L, uc, cand);
                hp.predicted_ms[b][L] = 1e3 * t;
                if (best < 0.0 || t < best) {
                    best = t;
                    bb = b;
                    bl = L;
                    // the plan's tree: everything build_tree writes
                    hp.src_perm = std::move(cand.src_perm);
                    hp.tgt_perm = std::move(cand.tgt_perm);
                    hp.levels = std::move(cand.levels);
                    hp.leaf_level = std::move(cand.leaf_level);
                    hp.leaf_box = std::move(cand.leaf_box);
                    hp.src_start = std::move(cand.src_start);
                    hp.src_count = std::move(cand.src_count);
                    hp.tgt_start = std::move(cand.tgt_start);
                    hp.tgt_count = std::move(cand.tgt_count);
                    hp.noff = std::move(cand.noff);
                    hp.nidx = std::move(cand.nidx);
                    hp.p2p_pairs = cand.p2p_pairs;
                    hp.p2p_self_pairs = cand.p2p_self_pairs;
                    hp.tree_ready = 1;
                }
            }
        }
    }
    hp.buffer = bb;
    hp.lp = lps[bb];
    hp.lf = lfb[bb] >= 2 ? bl : lfb[bb];
    hp.tuned = lfb[bb] >= 2 ? 1 : 0;
    if (hp.lf < lfb[bb]) hp.occ_depth = hp.lf;   // capped below the deepest stable level
}

// ---------------------------------------------------------------------------
std::string build_host_plan(HostPlan& hp) {
    alloc_point();
    // root cube
    std::vector<double> lo(3), hi(3);
    for (int k = 0; k < 3; ++k) {
        lo[k] = hp.src[k];
        hi[k] = hp.src[k];
    }
    for (int64_t i = 0; i < hp.ns; ++i)
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], hp.src[3 * i + k]);
            hi[k] = std::max(hi[k], hp.src[3 * i + k]);
        }
    for (int64_t i = 0; i < hp.nt; ++i)
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], hp.tgt[3 * i + k]);
            hi[k] = std::max(hi[k], hp.tgt[3 * i + k]);
        }
    if (hp.has_root) {
        for (int k = 0; k < 3; ++k) hp.corner[k] = hp.root[k];
        hp.side = hp.root[3];
    } else {
        double side = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
        if (side == 0.0) side = 1.0;
        hp.side = side;
        for (int k = 0; k < 3; ++k) hp.corner[k] = (lo[k] + hi[k]) / 2.0 - side / 2.0;
    }
    // sorted depth-kTreeBits keys of the sources and targets (occupancy rule, plan-shape tuner)
    std::vector<uint64_t> ks, kt;
    const bool same = hp.ns == hp.nt && hp.src == hp.tgt;
    if (hp.depth_req == 0 || hp.buffer == 0) {
        leaf_keys(hp.src, hp.ns, hp.corner, hp.side, ks);
        psort(ks);
        if (same) {
            kt = ks;
        } else {
            leaf_keys(hp.tgt, hp.nt, hp.corner, hp.side, kt);
            psort(kt);
        }
    }
    alloc_point();
    // depth bound
    if (hp.depth_req > 0) {
        hp.occ_depth = hp.depth_req;
    } else {
        hp.occ_depth = kTreeBits;
        for (int d = 0; d <= kTreeBits; ++d) {
            int sh = 3 * (kTreeBits - d);
            if (max_run(ks, sh) <= hp.max_leaf && max_run(kt, sh) <= hp.max_leaf) {
                hp.occ_depth = d;
                break;
            }
        }
    }
    hp.eps_l = hp.eps_scale * hp.eps;
    alloc_point();
    if (hp.buffer == 0) {
        tune_plan_shape(hp, ks, kt);
    } else {
        hp.lp = plan_levels(hp, hp.buffer, hp.occ_depth, &hp.lf);
    }
    // the device transforms work on lengths up to 1024: refuse before the costly tables
    for (int l = 2; l <= hp.lf; ++l) {
        if (hp.lp[l].quad.ntheta > 1024) return "N_theta above 1024 is not supported";
        for (int v : hp.lp[l].quad.nphi)
            if (v > 1024) return "N_phi above 1024 is not supported";
    }
    alloc_point();
    if (!hp.tree_ready) build_tree(hp);
    for (int l = 2; l <= hp.lf && hp.host_tables; ++l) {
        alloc_point();
        std::vector<char> used(transfer_slots(hp.buffer), 0);
        for (int32_t v : hp.levels[l].iv) used[v] = 1;
        build_tables(hp.lp[l], hp.kappa, hp.buffer, used);
    }
    return "";
}

}  // namespace hfmm
