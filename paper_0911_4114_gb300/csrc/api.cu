// C ABI of the GB300 Fourier-basis Helmholtz FMM (declared in include/hfmm.h):
// plan creation (host planner + one upload), the device apply and the queries.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <type_traits>
#include <utility>
#include <string>
#include <vector>

#include "../../include/hfmm.h"
#include "host_plan.hpp"
#include "kernels.cuh"
#include "tc5.cuh"

using namespace hfmm;

namespace {

thread_local std::string g_err;
// allocation points left before the planner's next one fails (hfmm_debug_fail_host_alloc)
thread_local int g_fail_alloc_after = -1;

hfmm_status fail(hfmm_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

}  // namespace

void hfmm::set_last_error(const std::string& msg) { g_err = msg; }

void hfmm::alloc_point() {
    if (g_fail_alloc_after < 0) return;
    if (g_fail_alloc_after-- == 0) throw std::bad_alloc();
}

namespace {

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(HFMM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

struct DevLevel {
    int prec = kFP64;
    int64_t K = 0;
    int nbox = 0;
    QuadView qv{};
    BoxView bv{};
    int32_t* octant = nullptr;
    // M2L by sibling groups (k_m2l_sib): parents at level l-1 with their first child and child
    // count, and per parent the union of the children's lists (box, child mask, slot per child
    // for the forward and the transposed M2L)
    std::vector<int32_t> slot_host;   // compact table slot of every transfer vector
    // M2L per box (k_m2l_box): CSR lists with the table slot of every entry (forward, transposed)
    int32_t *ioff = nullptr, *iidx = nullptr, *islot = nullptr, *islot_t = nullptr;
    bool m2l_sib = false;             // M2L kernel the plan timed faster on this level
    int npar = 0;
    int32_t *pfirst = nullptr, *pnch = nullptr, *poff = nullptr, *pu = nullptr, *pmask = nullptr;
    int32_t *pslot = nullptr, *pslot_t = nullptr;
    void* table = nullptr;      // compact T^{s,LL} tables in the level precision
    df* sdf = nullptr;          // (K, 3) s_k * kappa / 2 pi as double-float pairs
    cxd* shift64 = nullptr;     // [8][K] exp(i k s.d_o), d_o = child-centre offsets of level l+1
    cxf* shift32 = nullptr;
    cx<df>* shiftdf = nullptr;
    void* M = nullptr;          // nbox * Rmax * K
    void* IL = nullptr;         // incoming, then local expansions (in place)
    // this level's leaves (a uniform tree's level-lf leaves are all its boxes, other levels
    // none): count, positions (null: every box), subtree point ranges per box, 32-point chunks
    // (box, first point) of the leaves' targets and sources, largest leaf point counts
    int nleaf = 0;
    const int32_t* leaf = nullptr;
    const int32_t *sstart = nullptr, *scount = nullptr, *tstart = nullptr, *tcount = nullptr;
    const int2 *tunits = nullptr, *sunits = nullptr;
    int ntunits = 0, nsunits = 0;
    int max_src = 1, max_tgt = 1;
};

struct Requad {
    RequadArgs args{};
    int64_t ga_elems = 0, gb_elems = 0;
    // pass B' as a dense product (k_requad_theta_dense) for short circles: the 2 x 2 blocks
    // (Lee, Leo, Loe, Loo)[n][u], nrb x nra, or null
    const float4* theta_w = nullptr;
    int nra = 0, nrb = 0;
    const float4* theta_wt = nullptr;   // the transposed pass (k_requad_spec_cols_t), nra x nrb
};

}  // namespace

struct hfmm_plan_s {
    HostPlan hp;
    int device = -1;
    // near-field arithmetic (kFP32 / kDF / kFP64).  The float32 exact-grid form carries ~1e-7
    // relative error per pair, double-float ~1e-13: the mixed policy takes float32 for
    // eps >= 1e-6, double-float for 1e-11 <= eps < 1e-6, float64 below; the float64 policy
    // always float64
    int near_prec = kFP64;
    // sources and targets are the same point set: the float32 near field evaluates each
    // pair of distinct neighbouring boxes once for both directions (one RHS)
    bool sym = false;
    // right-hand sides from which the float32 near field runs as a tensor-core GEMM form
    static constexpr int kTcMinRhs = 8;
    df* tpos_df = nullptr;      // (nt, 3) sorted targets minus the root corner, double-float
    df* spos_df = nullptr;      // (ns, 3) sorted sources
    int rmax = 1;
    std::vector<void*> allocs;
    // leaf / points
    int64_t *src_perm = nullptr, *tgt_perm = nullptr;
    double *sx = nullptr, *sy = nullptr, *sz = nullptr, *tx = nullptr, *ty = nullptr, *tz = nullptr;
    int32_t *sstart = nullptr, *scount = nullptr, *tstart = nullptr, *tcount = nullptr;
    int32_t *noff = nullptr, *nidx = nullptr;
    P2PMixedArgs mixed{};
    cxd *qs = nullptr, *phis = nullptr;
    int max_src_leaf = 1, max_tgt_leaf = 1;   // largest leaf-box point counts (grid heights)
    int2 *tunits = nullptr, *sunits = nullptr;  // (leaf box, first point) of every 32-point chunk
    int ntunits = 0, nsunits = 0;
    int2* symunits = nullptr;                   // the same chunks, heaviest first (symmetric near field)
    int nsymunits = 0;
    int sym_variant = 7;      // resident-block target of the symmetric near-field kernel (tuned)
    int2 *tunits64 = nullptr, *sunits64 = nullptr;  // 64-point chunks (tensor-core near field)
    int ntunits64 = 0, nsunits64 = 0;
    // right-hand sides from which the float32 near field runs on tcgen05 (k_p2p_tc5)
    static constexpr int kTc5MinRhs = 16;
    // tcgen05 near field, per side (s: sources, t: targets): 16-point tiles of every leaf box
    // (first sorted point, count); per direction the units (box, first point of a 128-chunk,
    // tiles over the neighbour list of the other side) grouped per CTA with their tile records
    int32_t *t5first_s = nullptr, *t5n_s = nullptr;
    int32_t *t5first_t = nullptr, *t5n_t = nullptr;
    int t5ntiles_s = 0, t5ntiles_t = 0;
    struct T5Dir {            // one direction (forward: target chunks; adjoint: source chunks)
        int4* units = nullptr;
        int32_t *cta_off = nullptr, *rec_off = nullptr;
        int2* recs = nullptr;
        int ncta = 0;
    } t5fwd, t5adj;
    int64_t t5tiles_fwd = 0;  // (chunk, tile) pairs of the forward direction per 64-RHS pass
    unsigned char* t5blk = nullptr;   // split charge operands, (tile, 64-RHS pass) blocks
    // device flag set by a kernel whose bounded wait gave up (read by hfmm_query)
    int* dev_err = nullptr;
    double* gsort = nullptr;    // sorted position gradient (ns, 3)
    DevLevel lev[kMaxLevels];
    Requad up[kMaxLevels];    // up[l]: level l -> l-1
    Requad down[kMaxLevels];  // down[l]: level l -> l+1
    void *ga = nullptr, *gb = nullptr;
    void *tw64 = nullptr, *tw32 = nullptr, *twdf = nullptr;
    int* twoff = nullptr;
    cdf* cis_tab = nullptr;     // exp(2 pi i j / 1024) as double-float pairs
    // plane-wave tables of a float64 leaf level: [sorted point][antipodal pair] (sources, and
    // targets unless the two point sets are the same); null when not built
    int64_t tab_budget = -1;
    cxd *tab_s = nullptr, *tab_t = nullptr;
    int64_t tab_bytes = 0;
    int64_t workspace = 0;
    bool timing = false;
    cudaEvent_t ev[HFMM_N_STAGES + 1] = {};
    bool ev_recorded = false;
};

namespace {

template <typename T>
hfmm_status dalloc(hfmm_plan_s* p, T** ptr, size_t count) {
    *ptr = nullptr;
    if (count == 0) count = 1;
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, count * sizeof(T));
    if (e != cudaSuccess) return fail(HFMM_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    p->allocs.push_back(v);
    p->workspace += (int64_t)(count * sizeof(T));
    *ptr = static_cast<T*>(v);
    return HFMM_OK;
}

template <typename T>
hfmm_status upload(hfmm_plan_s* p, T** ptr, const std::vector<T>& host) {
    hfmm_status s = dalloc(p, ptr, host.size());
    if (s != HFMM_OK) return s;
    if (!host.empty()) CK(cudaMemcpy(*ptr, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice));
    return HFMM_OK;
}

#define TRY(x)                          \
    do {                                \
        hfmm_status s_ = (x);           \
        if (s_ != HFMM_OK) return s_;   \
    } while (0)

size_t cx_bytes(int prec) { return prec == kFP32 ? sizeof(cxf) : sizeof(cxd); }

hfmm_status upload_level(hfmm_plan_s* P, int l) {
    HostPlan& hp = P->hp;
    DevLevel& d = P->lev[l];
    const TreeLevel& T = hp.levels[l];
    const LevelPlan& lp = hp.lp[l];
    const Quadrature& q = lp.quad;
    d.prec = lp.prec;
    d.K = q.K;
    d.nbox = (int)T.nbox();
    // quadrature
    std::vector<double> shat(3 * q.K), w(q.K);
    const int half = q.ntheta / 2;
    const double two_pi = 2.0 * 3.14159265358979323846;
    for (int n = 0; n <= half; ++n) {
        const double th = two_pi * n / q.ntheta;
        const int np = q.nphi[n];
        const double mult = (n == 0 || n == half) ? 1.0 : 2.0;
        for (int m = 0; m < np; ++m) {
            const double ph = two_pi * m / np;
            const int64_t k = q.off[n] + m;
            shat[3 * k] = std::cos(ph) * std::sin(th);
            shat[3 * k + 1] = std::sin(ph) * std::sin(th);
            shat[3 * k + 2] = std::cos(th);
            w[k] = mult * (two_pi * two_pi) / ((double)q.ntheta * (double)np);
        }
    }
    int* nphi;
    int64_t* off;
    double *dshat, *dw;
    TRY(upload(P, &nphi, q.nphi));
    TRY(upload(P, &off, q.off));
    TRY(upload(P, &dshat, shat));
    TRY(upload(P, &dw, w));
    // antipodal pairs: (n, m) with n < N_theta/2 - n, or the middle row's first half
    std::vector<int2> pairs;
    pairs.reserve(q.K / 2);
    for (int n = 0; 2 * n <= half; ++n) {
        const int np = q.nphi[n];
        if (np % 2 != 0 || q.nphi[half - n] != np)
            return fail(HFMM_ERR_STATE, "quadrature grid is not antipodally symmetric");
        const int mend = (2 * n == half) ? np / 2 : np;
        for (int m = 0; m < mend; ++m)
            pairs.push_back(make_int2((int)(q.off[n] + m), (int)(q.off[half - n] + (m + np / 2) % np)));
    }
    if ((int64_t)pairs.size() * 2 != q.K) return fail(HFMM_ERR_STATE, "antipodal pairs do not cover the grid");
    int2* dpair;
    TRY(upload(P, &dpair, pairs));
    std::vector<float> asp(6 * q.K);
    {
        const double kt = hp.kappa / (2.0 * 3.14159265358979323846);
        for (int64_t k = 0; k < q.K; ++k)
            for (int c = 0; c < 3; ++c) {
                const double a = kt * shat[3 * k + c];
                asp[6 * k + c] = (float)a;
                asp[6 * k + 3 + c] = (float)(a - (double)(float)a);
            }
    }
    float* dasp;
    TRY(upload(P, &dasp, asp));
    d.qv = QuadView{q.ntheta, half + 1, q.K, nphi, off, dshat, dw, dpair, (int64_t)pairs.size(), dasp};
    {
        std::vector<df> sd(3 * q.K);
        const double kt = hp.kappa / (2.0 * 3.14159265358979323846);
        for (int64_t i = 0; i < 3 * q.K; ++i) sd[i] = df_from_double(shat[i] * kt);
        TRY(upload(P, &d.sdf, sd));
    }
    // boxes
    double* center;
    int32_t *idx, *parent, *cs = nullptr, *cc = nullptr;
    TRY(upload(P, &center, T.center));
    TRY(upload(P, &idx, T.idx));
    TRY(upload(P, &parent, T.parent));
    if (!T.child_start.empty()) {
        TRY(upload(P, &cs, T.child_start));
        TRY(upload(P, &cc, T.child_count));
    }
    d.bv = BoxView{d.nbox, center, idx, parent, cs, cc};
    // leaves of this level
    if (!hp.adaptive) {
        if (l == hp.lf) {
            d.nleaf = d.nbox;
            d.sstart = P->sstart;
            d.scount = P->scount;
            d.tstart = P->tstart;
            d.tcount = P->tcount;
            d.tunits = P->tunits;
            d.sunits = P->sunits;
            d.ntunits = P->ntunits;
            d.nsunits = P->nsunits;
            d.max_src = P->max_src_leaf;
            d.max_tgt = P->max_tgt_leaf;
        }
    } else if (!T.leaf_pos.empty()) {
        d.nleaf = (int)T.leaf_pos.size();
        int32_t *lp_, *ss, *sc, *ts, *tc;
        TRY(upload(P, &lp_, T.leaf_pos));
        TRY(upload(P, &ss, T.s_start));
        TRY(upload(P, &sc, T.s_count));
        TRY(upload(P, &ts, T.t_start));
        TRY(upload(P, &tc, T.t_count));
        d.leaf = lp_;
        d.sstart = ss;
        d.scount = sc;
        d.tstart = ts;
        d.tcount = tc;
        std::vector<int2> tu, su;
        for (int32_t b : T.leaf_pos) {
            for (int c = 0; c < T.t_count[b]; c += 32) tu.push_back(make_int2(b, c));
            for (int c = 0; c < T.s_count[b]; c += 32) su.push_back(make_int2(b, c));
            d.max_src = std::max(d.max_src, (int)T.s_count[b]);
            d.max_tgt = std::max(d.max_tgt, (int)T.t_count[b]);
        }
        int2 *dtu, *dsu;
        TRY(upload(P, &dtu, tu));
        TRY(upload(P, &dsu, su));
        d.tunits = dtu;
        d.sunits = dsu;
        d.ntunits = (int)tu.size();
        d.nsunits = (int)su.size();
    }
    std::vector<int32_t> oct(d.nbox);
    for (int b = 0; b < d.nbox; ++b)
        oct[b] = 4 * (T.idx[3 * b] & 1) + 2 * (T.idx[3 * b + 1] & 1) + (T.idx[3 * b + 2] & 1);
    TRY(upload(P, &d.octant, oct));
    // transfer tables, compact: slot of every used vector (the lists are symmetric, so the
    // opposite vector W^3 - 1 - v of a used v is used too; the transposed M2L takes its slot)
    const int nslots = transfer_slots(hp.buffer);
    std::vector<char> used(nslots, 0);
    for (int32_t v : T.iv) used[v] = 1;
    std::vector<int32_t> slot(nslots, 0);
    int ns = 0;
    for (int v = 0; v < nslots; ++v) slot[v] = used[v] ? ns++ : 0;
    std::vector<int32_t> slot_t(nslots, 0);
    for (int v = 0; v < nslots; ++v) slot_t[v] = slot[nslots - 1 - v];
    d.slot_host = slot;
    {
        std::vector<int32_t> es(T.iv.size()), est(T.iv.size());
        for (size_t t = 0; t < T.iv.size(); ++t) {
            es[t] = slot[T.iv[t]];
            est[t] = slot_t[T.iv[t]];
        }
        TRY(upload(P, &d.ioff, T.ioff));
        TRY(upload(P, &d.iidx, T.iidx));
        TRY(upload(P, &d.islot, es));
        TRY(upload(P, &d.islot_t, est));
    }
    {
        // sibling groups: the children of each parent are contiguous at this level
        const TreeLevel& PL = hp.levels[l - 1];
        std::vector<int32_t> pf, pn, po(1, 0), pu, pm, ps, pst;
        std::vector<int32_t> mark(d.nbox, -1);
        for (int64_t pp = 0; pp < PL.nbox(); ++pp) {
            const int c0 = PL.child_start[pp], nc = PL.child_count[pp];
            if (nc == 0) continue;
            if (nc > 8) return fail(HFMM_ERR_STATE, "internal: more than 8 children");
            pf.push_back(c0);
            pn.push_back(nc);
            // union of the children's lists, in box order (= Morton order)
            std::vector<int32_t> us;
            for (int c = 0; c < nc; ++c)
                for (int32_t t = T.ioff[c0 + c]; t < T.ioff[c0 + c + 1]; ++t) us.push_back(T.iidx[t]);
            std::sort(us.begin(), us.end());
            us.erase(std::unique(us.begin(), us.end()), us.end());
            const size_t base = pu.size();
            for (size_t i = 0; i < us.size(); ++i) mark[us[i]] = (int32_t)(base + i);
            pu.insert(pu.end(), us.begin(), us.end());
            pm.resize(pu.size(), 0);
            ps.resize(8 * pu.size(), 0);
            pst.resize(8 * pu.size(), 0);
            for (int c = 0; c < nc; ++c)
                for (int32_t t = T.ioff[c0 + c]; t < T.ioff[c0 + c + 1]; ++t) {
                    const int32_t e = mark[T.iidx[t]];
                    pm[e] |= 1 << c;
                    ps[8 * (size_t)e + c] = slot[T.iv[t]];
                    pst[8 * (size_t)e + c] = slot_t[T.iv[t]];
                }
            po.push_back((int32_t)pu.size());
        }
        d.npar = (int)pf.size();
        TRY(upload(P, &d.pfirst, pf));
        TRY(upload(P, &d.pnch, pn));
        TRY(upload(P, &d.poff, po));
        TRY(upload(P, &d.pu, pu));
        TRY(upload(P, &d.pmask, pm));
        TRY(upload(P, &d.pslot, ps));
        TRY(upload(P, &d.pslot_t, pst));
    }
    if (!hp.host_tables) {
        // T^{s,LL} on the device (tables.cu), in the level's storage
        void* dt = nullptr;
        size_t bytes = 0;
        const std::string e = device_tables(make_table_job(lp, hp.kappa, hp.buffer, used), q,
                                            d.prec == kFP32 ? 0 : (d.prec == kFP64 ? 1 : 2), &dt, &bytes);
        if (!e.empty()) return fail(HFMM_ERR_CUDA, e);
        if (dt) {
            P->allocs.push_back(dt);
            P->workspace += (int64_t)bytes;
        }
        d.table = dt;
    } else if (d.prec == kDF) {
        std::vector<cx<df>> t((size_t)ns * q.K);
        for (int v = 0; v < transfer_slots(hp.buffer); ++v)
            if (!lp.table[v].empty())
                for (int64_t k = 0; k < q.K; ++k)
                    t[(size_t)slot[v] * q.K + k] = mk<df>(df(lp.table[v][k].real()), df(lp.table[v][k].imag()));
        cx<df>* dt;
        TRY(upload(P, &dt, t));
        d.table = dt;
    } else if (d.prec == kFP64) {
        std::vector<cxd> t((size_t)ns * q.K);
        for (int v = 0; v < transfer_slots(hp.buffer); ++v)
            if (!lp.table[v].empty())
                for (int64_t k = 0; k < q.K; ++k)
                    t[(size_t)slot[v] * q.K + k] = mk<double>(lp.table[v][k].real(), lp.table[v][k].imag());
        cxd* dt;
        TRY(upload(P, &dt, t));
        d.table = dt;
    } else {
        std::vector<cxf> t((size_t)ns * q.K);
        for (int v = 0; v < transfer_slots(hp.buffer); ++v)
            if (!lp.table[v].empty())
                for (int64_t k = 0; k < q.K; ++k)
                    t[(size_t)slot[v] * q.K + k] =
                        mk<float>((float)lp.table[v][k].real(), (float)lp.table[v][k].imag());
        cxf* dt;
        TRY(upload(P, &dt, t));
        d.table = dt;
    }
    // shift tables for the child offsets of level l+1 (M2M into l, L2L out of l)
    if (l < hp.lf) {
        const double ac = hp.side / (double)(1u << (l + 1));
        std::vector<cxd> s64((size_t)8 * q.K);
        std::vector<cxf> s32((size_t)8 * q.K);
        std::vector<cx<df>> sdf((size_t)8 * q.K);
        for (int o = 0; o < 8; ++o) {
            const double dvec[3] = {(((o >> 2) & 1) - 0.5) * ac, (((o >> 1) & 1) - 0.5) * ac,
                                    ((o & 1) - 0.5) * ac};
            for (int64_t k = 0; k < q.K; ++k) {
                const double ph = hp.kappa * (shat[3 * k] * dvec[0] + shat[3 * k + 1] * dvec[1] +
                                              shat[3 * k + 2] * dvec[2]);
                s64[(size_t)o * q.K + k] = mk<double>(std::cos(ph), std::sin(ph));
                s32[(size_t)o * q.K + k] = mk<float>((float)std::cos(ph), (float)std::sin(ph));
                sdf[(size_t)o * q.K + k] = mk<df>(df(std::cos(ph)), df(std::sin(ph)));
            }
        }
        TRY(upload(P, &d.shift64, s64));
        TRY(upload(P, &d.shift32, s32));
        TRY(upload(P, &d.shiftdf, sdf));
    }
    // signature buffers
    const size_t bytes = (size_t)d.nbox * P->rmax * q.K * cx_bytes(d.prec);
    unsigned char *m, *il;
    TRY(dalloc(P, &m, bytes));
    TRY(dalloc(P, &il, bytes));
    d.M = m;
    d.IL = il;
    return HFMM_OK;
}

Requad make_requad(const Quadrature& a, const Quadrature& b, int nbox_seq, int rmax) {
    Requad r;
    int big = 0;
    for (int v : a.nphi) big = std::max(big, v);
    for (int v : b.nphi) big = std::max(big, v);
    r.args.big = big;
    r.args.maxlen = std::max(big, std::max(a.ntheta, b.ntheta));
    r.ga_elems = (int64_t)nbox_seq * rmax * (a.ntheta / 2 + 1) * big;
    r.gb_elems = (int64_t)nbox_seq * rmax * (b.ntheta / 2 + 1) * big;
    return r;
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// The theta pass of k_requad_spec_cols for one coefficient pair as matrices, in float64: the
// even circle of column u (rows 0 .. nta/2 of the grid a) is 1 at t = u and t = nta - u, the
// odd one +1 at t = u and -1 at t = nta - u (t > nta/2); each is band-limited re-sampled to
// length ntb (forward DFT, |f| <= min(ceil(nta/2), ceil(ntb/2)) - 1, 1/nta, inverse DFT) and
// split into its even (y[n] + y[-n]) / 2 and odd (y[n] - y[-n]) / 2 parts, n = 0 .. ntb/2.
// Entry n * nra + u: (even part of the even circle, of the odd circle; odd part of the even
// circle, of the odd circle).
// The transposed theta pass (k_requad_spec_cols_t, rows n of grid b -> rows u of grid a) the
// same way: unit values at row n of the even slot spread half onto m = n and m = ntb - n (the
// whole value at n = 0 and n = ntb/2), of the odd slot +-half (nothing at n = 0, ntb/2); the
// circle is re-sampled from ntb to nta (1/ntb), row u collects t = u and t = nta - u (the odd
// slot with a sign flip), scaled by ntb / nta.  Entry u * nrb + n as in theta_matrices.
std::vector<float4> theta_matrices_t(int nta, int ntb) {
    const int ha = nta / 2, hbr = ntb / 2, nra = ha + 1, nrb = hbr + 1;
    const int band = std::min((nta + 1) / 2, (ntb + 1) / 2) - 1;
    const double two_pi = 2.0 * 3.14159265358979323846, sc = (double)ntb / nta;
    auto resample = [&](const std::vector<std::pair<int, double>>& y, int t) {
        double r = 0.0;
        for (int f = -band; f <= band; ++f)
            for (const auto& mv : y) r += mv.second * std::cos(two_pi * f * ((double)t / nta - (double)mv.first / ntb));
        return r / ntb;
    };
    std::vector<float4> w((size_t)nra * nrb);
    for (int n = 0; n < nrb; ++n) {
        std::vector<std::pair<int, double>> ev, od;
        if (n == 0 || n == hbr) {
            ev.push_back({n, 1.0});
        } else {
            ev = {{n, 0.5}, {ntb - n, 0.5}};
            od = {{n, 0.5}, {ntb - n, -0.5}};
        }
        for (int u = 0; u < nra; ++u) {
            const bool two = u != 0 && u != ha;
            const double e0 = resample(ev, u), em = two ? resample(ev, nta - u) : 0.0;
            const double o0 = od.empty() ? 0.0 : resample(od, u), om = (two && !od.empty()) ? resample(od, nta - u) : 0.0;
            w[(size_t)u * nrb + n] = make_float4((float)(sc * (e0 + em)), (float)(sc * (o0 + om)), (float)(sc * (e0 - em)),
                                                 (float)(sc * (o0 - om)));
        }
    }
    return w;
}

std::vector<float4> theta_matrices(int nta, int ntb) {
    const int ha = nta / 2, nra = ha + 1, nrb = ntb / 2 + 1;
    const int band = std::min((nta + 1) / 2, (ntb + 1) / 2) - 1;
    const double two_pi = 2.0 * 3.14159265358979323846;
    auto resample = [&](const std::vector<std::pair<int, double>>& x, int m) {
        double y = 0.0;
        for (int f = -band; f <= band; ++f)
            for (const auto& tv : x) y += tv.second * std::cos(two_pi * f * ((double)m / ntb - (double)tv.first / nta));
        return y / nta;
    };
    std::vector<float4> w((size_t)nrb * nra);
    for (int u = 0; u < nra; ++u) {
        std::vector<std::pair<int, double>> ev{{u, 1.0}}, od{{u, 1.0}};
        if (u != 0 && u != ha) {
            ev.push_back({nta - u, 1.0});
            od.push_back({nta - u, -1.0});
        }
        for (int n = 0; n < nrb; ++n) {
            const int mn = (ntb - n) % ntb;
            const double ye = resample(ev, n), yem = resample(ev, mn), yo = resample(od, n), yom = resample(od, mn);
            w[(size_t)n * nra + u] = make_float4((float)(0.5 * (ye + yem)), (float)(0.5 * (yo + yom)),
                                                 (float)(0.5 * (ye - yem)), (float)(0.5 * (yo - yom)));
        }
    }
    return w;
}

// Plane-wave tables of a float64 leaf level (see k_pw_table), when they fit the budget.
hfmm_status build_leaf_tables(hfmm_plan_s* P) {
    const HostPlan& hp = P->hp;
    const int lf = hp.lf;
    if (lf < 2 || P->lev[lf].prec != kFP64 || P->tab_budget == 0) return HFMM_OK;
    const DevLevel& d = P->lev[lf];
    const int64_t npair = d.qv.npair;
    const int64_t rows = hp.ns + (P->sym ? 0 : hp.nt);
    const int64_t bytes = rows * npair * (int64_t)sizeof(cxd);
    int64_t budget = P->tab_budget;
    if (budget < 0) {
        size_t fr = 0, tot = 0;
        CK(cudaMemGetInfo(&fr, &tot));
        budget = (int64_t)(fr / 2);
    }
    if (bytes > budget) return HFMM_OK;
    const double kt = hp.kappa / (2.0 * 3.14159265358979323846);
    TRY(dalloc(P, &P->tab_s, (size_t)hp.ns * npair));
    if (P->nsunits > 0)
        k_pw_table<<<dim3(P->nsunits, nblk(npair, kTabThreads)), kTabThreads>>>(P->sunits, d.bv, d.qv, P->sstart,
                                                                               P->scount, P->sx, P->sy, P->sz, kt,
                                                                               P->tab_s);
    if (P->sym) {
        P->tab_t = P->tab_s;
    } else {
        TRY(dalloc(P, &P->tab_t, (size_t)hp.nt * npair));
        if (P->ntunits > 0)
            k_pw_table<<<dim3(P->ntunits, nblk(npair, kTabThreads)), kTabThreads>>>(
                P->tunits, d.bv, d.qv, P->tstart, P->tcount, P->tx, P->ty, P->tz, kt, P->tab_t);
    }
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    P->tab_bytes = bytes;
    return HFMM_OK;
}

// tcgen05 near field (k_p2p_tc5): the 16-point tiles of both sides, the units of both
// directions dealt round robin in Morton order to one persistent CTA per SM, and the
// split-charge block buffer for max_rhs right-hand sides.  Round robin keeps the units that
// the CTAs work on at one time next to each other, so their neighbour lists, and the charge
// blocks they read, largely coincide (the blocks are then read from L2)
hfmm_status build_t5(hfmm_plan_s* P) {
    HostPlan& hp = P->hp;
    int nsm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, P->device));
    nsm = std::max(nsm, 1);
    auto tiles = [&](const std::vector<int32_t>& start, const std::vector<int32_t>& count, std::vector<int32_t>& base,
                     int32_t** dfirst, int32_t** dn, int* ntiles) -> hfmm_status {
        std::vector<int32_t> first, n;
        base.assign(count.size(), 0);
        for (size_t b = 0; b < count.size(); ++b) {
            base[b] = (int32_t)first.size();
            for (int c = 0; c < count[b]; c += kT5Src) {
                first.push_back(start[b] + c);
                n.push_back(std::min(kT5Src, count[b] - c));
            }
        }
        if (first.size() >= (size_t(1) << 27)) return fail(HFMM_ERR_ARG, "too many near-field tiles");
        *ntiles = (int)first.size();
        TRY(upload(P, dfirst, first));
        TRY(upload(P, dn, n));
        return HFMM_OK;
    };
    std::vector<int32_t> sbase, tbase;
    TRY(tiles(hp.src_start, hp.src_count, sbase, &P->t5first_s, &P->t5n_s, &P->t5ntiles_s));
    TRY(tiles(hp.tgt_start, hp.tgt_count, tbase, &P->t5first_t, &P->t5n_t, &P->t5ntiles_t));
    // units of one side (128-point chunks of its boxes) dealt round robin, and for every unit
    // the records of the other side's tiles over its neighbour list
    auto sched = [&](const std::vector<int32_t>& ucount, const std::vector<int32_t>& ostart,
                     const std::vector<int32_t>& ocount, const std::vector<int32_t>& obase, hfmm_plan_s::T5Dir* d) -> hfmm_status {
        std::vector<int4> u;
        for (size_t b = 0; b < ucount.size(); ++b) {
            int nt = 0;
            for (int32_t t = hp.noff[b]; t < hp.noff[b + 1]; ++t) nt += (ocount[hp.nidx[t]] + kT5Src - 1) / kT5Src;
            for (int c = 0; c < ucount[b]; c += kT5M) u.push_back(make_int4((int)b, c, nt, 0));
        }
        const int nc = std::max(1, std::min(nsm, (int)u.size()));
        std::vector<std::vector<int4>> bins(nc);
        for (size_t k = 0; k < u.size(); ++k) bins[k % nc].push_back(u[k]);
        std::vector<int4> flat;
        std::vector<int32_t> off(1, 0), roff;
        std::vector<int2> recs;
        for (const auto& bin : bins) {
            for (const int4& x : bin) {
                if (recs.size() + (size_t)x.z >= (size_t)INT32_MAX) return fail(HFMM_ERR_ARG, "too many near-field tiles");
                roff.push_back((int32_t)recs.size());
                for (int32_t t = hp.noff[x.x]; t < hp.noff[x.x + 1]; ++t) {
                    const int32_t s = hp.nidx[t];
                    for (int c = 0; c < ocount[s]; c += kT5Src) {
                        const int sn = std::min(kT5Src, ocount[s] - c);
                        recs.push_back(make_int2(ostart[s] + c, (obase[s] + c / kT5Src) | ((sn - 1) << 27)));
                    }
                }
                flat.push_back(x);
            }
            off.push_back((int32_t)flat.size());
        }
        d->ncta = nc;
        if (d == &P->t5fwd) P->t5tiles_fwd = (int64_t)recs.size();
        TRY(upload(P, &d->units, flat));
        TRY(upload(P, &d->cta_off, off));
        TRY(upload(P, &d->rec_off, roff));
        TRY(upload(P, &d->recs, recs));
        return HFMM_OK;
    };
    TRY(sched(hp.tgt_count, hp.src_start, hp.src_count, sbase, &P->t5fwd));
    TRY(sched(hp.src_count, hp.tgt_start, hp.tgt_count, tbase, &P->t5adj));
    const size_t npass = (size_t)(P->rmax + kT5Rhs - 1) / kT5Rhs;
    TRY(dalloc(P, &P->t5blk, (size_t)std::max(P->t5ntiles_s, P->t5ntiles_t) * npass * kT5Blk));
    return HFMM_OK;
}

// tcgen05 near field of one direction: split the charge operands, then the persistent kernel
// (forward: target chunks over source tiles, q -> phi; adjoint: source chunks over target
// tiles, w -> A^H w)
void launch_t5(hfmm_plan_s* P, bool adjoint, int R, cudaStream_t st) {
    const int npass = (R + kT5Rhs - 1) / kT5Rhs;
    const int ntiles = adjoint ? P->t5ntiles_t : P->t5ntiles_s;
    const cxd* in = adjoint ? P->phis : P->qs;
    if (ntiles > 0)
        k_t5_bsplit<<<(unsigned)((int64_t)ntiles * npass), 256, 0, st>>>(adjoint ? P->t5first_t : P->t5first_s,
                                                                         adjoint ? P->t5n_t : P->t5n_s, ntiles,
                                                                         npass, in, R, P->t5blk);
    const hfmm_plan_s::T5Dir& d = adjoint ? P->t5adj : P->t5fwd;
    T5Args g{};
    g.units = d.units;
    g.cta_off = d.cta_off;
    g.tstart = adjoint ? P->sstart : P->tstart;
    g.tcount = adjoint ? P->scount : P->tcount;
    g.rec_off = d.rec_off;
    g.recs = d.recs;
    g.bblk = P->t5blk;
    g.a = P->mixed;
    if (adjoint) {
        std::swap(g.a.tpt, g.a.spt);
        std::swap(g.a.tof, g.a.sof);
    }
    g.phis = adjoint ? P->qs : P->phis;
    g.R = R;
    g.err = P->dev_err;
    cudaFuncSetAttribute(k_p2p_tc5, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kT5Smem);
    k_p2p_tc5<<<d.ncta, kT5Threads, kT5Smem, st>>>(g);
}

hfmm_status upload_plan(hfmm_plan_s* P) {
    HostPlan& hp = P->hp;
    CK(cudaSetDevice(P->device));
    // points, sorted, SoA
    auto soa = [&](const std::vector<double>& pts, const std::vector<int64_t>& perm, double** x, double** y,
                   double** z) -> hfmm_status {
        std::vector<double> a(perm.size()), b(perm.size()), c(perm.size());
        for (size_t i = 0; i < perm.size(); ++i) {
            a[i] = pts[3 * perm[i]];
            b[i] = pts[3 * perm[i] + 1];
            c[i] = pts[3 * perm[i] + 2];
        }
        TRY(upload(P, x, a));
        TRY(upload(P, y, b));
        TRY(upload(P, z, c));
        return HFMM_OK;
    };
    TRY(soa(hp.src, hp.src_perm, &P->sx, &P->sy, &P->sz));
    TRY(soa(hp.tgt, hp.tgt_perm, &P->tx, &P->ty, &P->tz));
    TRY(upload(P, &P->src_perm, hp.src_perm));
    TRY(upload(P, &P->tgt_perm, hp.tgt_perm));
    {
        auto chunks = [&](const std::vector<int32_t>& count, int2** dst, int* n, int width) -> hfmm_status {
            std::vector<int2> u;
            for (size_t b = 0; b < count.size(); ++b)
                for (int c = 0; c < count[b]; c += width) u.push_back(make_int2((int)b, c));
            *n = (int)u.size();
            return upload(P, dst, u);
        };
        TRY(chunks(hp.tgt_count, &P->tunits, &P->ntunits, 32));
        TRY(chunks(hp.src_count, &P->sunits, &P->nsunits, 32));
        if (P->rmax >= hfmm_plan_s::kTcMinRhs) {
            TRY(chunks(hp.tgt_count, &P->tunits64, &P->ntunits64, 64));
            TRY(chunks(hp.src_count, &P->sunits64, &P->nsunits64, 64));
        }
        if (P->rmax >= hfmm_plan_s::kTc5MinRhs) TRY(build_t5(P));
        if (P->sym) {
            // symmetric near field: a unit of box b sums over neighbours s >= b, so the work of
            // units varies widely; launch them heaviest first (longest-processing-time order)
            std::vector<std::pair<int64_t, int2>> w;
            for (size_t b = 0; b < hp.tgt_count.size(); ++b) {
                int64_t work = 0;
                for (int32_t t = hp.noff[b]; t < hp.noff[b + 1]; ++t)
                    if (hp.nidx[t] >= (int32_t)b) work += hp.src_count[hp.nidx[t]];
                for (int c = 0; c < hp.tgt_count[b]; c += 32)
                    w.push_back({work * std::min(32, hp.tgt_count[b] - c), make_int2((int)b, c)});
            }
            std::stable_sort(w.begin(), w.end(), [](const std::pair<int64_t, int2>& a, const std::pair<int64_t, int2>& b) {
                return a.first > b.first;
            });
            std::vector<int2> u(w.size());
            for (size_t i = 0; i < w.size(); ++i) u[i] = w[i].second;
            P->nsymunits = (int)u.size();
            TRY(upload(P, &P->symunits, u));
        }

    }
    for (int32_t c : hp.src_count) P->max_src_leaf = std::max(P->max_src_leaf, (int)c);
    for (int32_t c : hp.tgt_count) P->max_tgt_leaf = std::max(P->max_tgt_leaf, (int)c);
    TRY(upload(P, &P->sstart, hp.src_start));
    TRY(upload(P, &P->scount, hp.src_count));
    TRY(upload(P, &P->tstart, hp.tgt_start));
    TRY(upload(P, &P->tcount, hp.tgt_count));
    TRY(upload(P, &P->noff, hp.noff));
    TRY(upload(P, &P->nidx, hp.nidx));
    // mixed-precision near-field geometry: exact grid integers + fractional offsets
    {
        const int gbits = std::min(12, 10 + std::max(0, hp.lf));
        const double cells = std::ldexp(1.0, gbits);
        const double scale = cells / hp.side;
        auto grid = [&](const std::vector<double>& pts, const std::vector<int64_t>& perm, const float4** g,
                        const float4** o) -> hfmm_status {
            // 16 zero points past the end: the tcgen05 near field copies whole 16-point tiles
            std::vector<float4> gg(perm.size() + 16, make_float4(0.f, 0.f, 0.f, 0.f)), oo(gg);
            for (size_t i = 0; i < perm.size(); ++i) {
                float gv[3], ov[3];
                for (int k = 0; k < 3; ++k) {
                    double u = (pts[3 * perm[i] + k] - hp.corner[k]) * scale;
                    double f = std::floor(u);
                    f = std::min(std::max(f, 0.0), cells - 1.0);
                    gv[k] = (float)f;
                    ov[k] = (float)(u - f);
                }
                gg[i] = make_float4(gv[0], gv[1], gv[2], 0.f);
                oo[i] = make_float4(ov[0], ov[1], ov[2], 0.f);
            }
            float4 *dg, *dof;
            TRY(upload(P, &dg, gg));
            TRY(upload(P, &dof, oo));
            *g = dg;
            *o = dof;
            return HFMM_OK;
        };
        TRY(grid(hp.tgt, hp.tgt_perm, &P->mixed.tpt, &P->mixed.tof));
        TRY(grid(hp.src, hp.src_perm, &P->mixed.spt, &P->mixed.sof));
        const double tau = hp.kappa * (hp.side / cells) / (2.0 * 3.14159265358979323846);
        P->mixed.tau_hi = (float)tau;
        P->mixed.tau_lo = (float)(tau - (double)P->mixed.tau_hi);
        P->mixed.inv_unit = scale;
        P->mixed.inv_unit_f = (float)scale;
    }
    if (P->near_prec == kDF) {
        auto pos = [&](const std::vector<double>& pts, const std::vector<int64_t>& perm, df** out) -> hfmm_status {
            std::vector<df> v(3 * perm.size());
            for (size_t i = 0; i < perm.size(); ++i)
                for (int k = 0; k < 3; ++k) v[3 * i + k] = df_from_double(pts[3 * perm[i] + k] - hp.corner[k]);
            return upload(P, out, v);
        };
        TRY(pos(hp.tgt, hp.tgt_perm, &P->tpos_df));
        TRY(pos(hp.src, hp.src_perm, &P->spos_df));
    }
    TRY(dalloc(P, &P->qs, (size_t)hp.ns * P->rmax));
    TRY(dalloc(P, &P->phis, (size_t)hp.nt * P->rmax));
    TRY(dalloc(P, &P->gsort, (size_t)hp.ns * 3));
    // levels
    for (int l = 2; l <= hp.lf; ++l) TRY(upload_level(P, l));
    // the re-quadrature dispatch covers precision pairs that never decrease with depth
    for (int l = 3; l <= hp.lf; ++l) {
        auto rank = [](int prec) { return prec == kFP32 ? 0 : (prec == kDF ? 1 : 2); };
        if (rank(P->lev[l].prec) < rank(P->lev[l - 1].prec))
            return fail(HFMM_ERR_STATE, "internal: level precision decreases with depth");
    }
    // re-quadrature passes and scratch
    int64_t ga = 0, gb = 0;
    std::vector<int> lengths;
    auto add_len = [&](const Quadrature& q) {
        for (int v : q.nphi) lengths.push_back(v);
        lengths.push_back(q.ntheta);
    };
    for (int l = 3; l <= hp.lf; ++l) {
        P->up[l] = make_requad(hp.lp[l].quad, hp.lp[l - 1].quad, P->lev[l].nbox, P->rmax);
        P->down[l - 1] = make_requad(hp.lp[l - 1].quad, hp.lp[l].quad, P->lev[l].nbox, P->rmax);
        for (auto rq : {std::make_pair(&P->up[l], std::make_pair(l, l - 1)), std::make_pair(&P->down[l - 1], std::make_pair(l - 1, l))}) {
            const int nta = hp.lp[rq.second.first].quad.ntheta, ntb = hp.lp[rq.second.second].quad.ntheta;
            if (nta / 2 + 1 <= kThetaDenseMax && ntb / 2 + 1 <= kThetaDenseMax) {
                float4* dw;
                TRY(upload(P, &dw, theta_matrices(nta, ntb)));
                rq.first->theta_w = dw;
                float4* dwt;
                TRY(upload(P, &dwt, theta_matrices_t(nta, ntb)));
                rq.first->theta_wt = dwt;
                rq.first->nra = nta / 2 + 1;
                rq.first->nrb = ntb / 2 + 1;
            }
        }
        for (Requad* r : {&P->up[l], &P->down[l - 1]}) {
            ga = std::max(ga, r->ga_elems);
            gb = std::max(gb, r->gb_elems);
            lengths.push_back(r->args.big);
        }
        add_len(hp.lp[l].quad);
        add_len(hp.lp[l - 1].quad);
    }
    TRY(dalloc(P, (cxd**)&P->ga, (size_t)ga));
    TRY(dalloc(P, (cxd**)&P->gb, (size_t)gb));
    // twiddle tables
    int maxlen = 1;
    for (int v : lengths) maxlen = std::max(maxlen, v);
    std::vector<int> off(maxlen + 1, -1);
    std::vector<cxd> t64;
    std::vector<cxf> t32;
    std::vector<cx<df>> tdf;
    std::sort(lengths.begin(), lengths.end());
    lengths.erase(std::unique(lengths.begin(), lengths.end()), lengths.end());
    for (int n : lengths) {
        if (!is_235(n)) return fail(HFMM_ERR_ARG, "internal: FFT length " + std::to_string(n) + " not 2^a3^b5^c");
        off[n] = (int)t64.size();
        for (int t = 0; t < n; ++t) {
            const double ang = 2.0 * 3.14159265358979323846 * (double)t / (double)n;
            t64.push_back(mk<double>(std::cos(ang), -std::sin(ang)));
            t32.push_back(mk<float>((float)std::cos(ang), (float)-std::sin(ang)));
            tdf.push_back(mk<df>(df(std::cos(ang)), df(-std::sin(ang))));
        }
    }
    cxd* d64;
    cxf* d32;
    cx<df>* ddf;
    TRY(upload(P, &d64, t64));
    TRY(upload(P, &d32, t32));
    TRY(upload(P, &ddf, tdf));
    TRY(upload(P, &P->twoff, off));
    P->tw64 = d64;
    P->tw32 = d32;
    P->twdf = ddf;
    for (int l = 2; l <= hp.lf; ++l) {
        for (Requad* r : {&P->up[l], &P->down[l]}) {
            r->args.tw.off = P->twoff;
        }
    }
    for (int l = 3; l <= hp.lf; ++l) {
        P->up[l].args.qa = P->lev[l].qv;
        P->up[l].args.qb = P->lev[l - 1].qv;
        P->down[l - 1].args.qa = P->lev[l - 1].qv;
        P->down[l - 1].args.qb = P->lev[l].qv;
    }
    {
        std::vector<cdf> tab(kCisTableBig);
        for (int j = 0; j < kCisTableBig; ++j) {
            const double a = 2.0 * 3.14159265358979323846 * (double)j / (double)kCisTableBig;
            tab[j] = cdf{df_from_double(std::cos(a)), df_from_double(std::sin(a))};
        }
        TRY(upload(P, &P->cis_tab, tab));
    }
    TRY(build_leaf_tables(P));
    TRY(dalloc(P, &P->dev_err, 1));
    CK(cudaMemset(P->dev_err, 0, sizeof(int)));
    for (int i = 0; i <= HFMM_N_STAGES; ++i) CK(cudaEventCreate(&P->ev[i]));
    return HFMM_OK;
}

// ---------------------------------------------------------------------------
// apply helpers
// ---------------------------------------------------------------------------

// opt a kernel into more than 48 KiB of dynamic shared memory when a launch needs it
template <typename K>
void smem_opt_in(K kernel, size_t bytes) {
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T> const void* pool_of(hfmm_plan_s* P);
template <> const void* pool_of<float>(hfmm_plan_s* P) { return P->tw32; }
template <> const void* pool_of<double>(hfmm_plan_s* P) { return P->tw64; }
template <> const void* pool_of<df>(hfmm_plan_s* P) { return P->twdf; }
template <typename T> const cx<T>* shift_of(const DevLevel& d);
template <> const cx<float>* shift_of<float>(const DevLevel& d) { return d.shift32; }
template <> const cx<double>* shift_of<double>(const DevLevel& d) { return d.shift64; }
template <> const cx<df>* shift_of<df>(const DevLevel& d) { return d.shiftdf; }

// pass B' (theta re-sampling) of a forward re-quadrature: the dense form for float32 short
// circles, else the warp-FFT form
template <typename Tc>
void launch_theta(const Requad& rq, const RequadArgs& ra, int nbox, int R, const cx<Tc>* GA, cx<Tc>* GB,
                  size_t sm, cudaStream_t st) {
    if (std::is_same<Tc, float>::value && rq.theta_w) {
        const int64_t nseq = (int64_t)nbox * R;
        const int64_t work = nseq * ra.big;
        const unsigned g = (unsigned)std::min<int64_t>((work + 127) / 128, 152 * 32);
        const int knr = rq.nra <= 9 ? 9 : (rq.nra <= 17 ? 17 : (rq.nra <= 25 ? 25 : 33));
        const size_t smw = (size_t)rq.nrb * knr * sizeof(float4);
        const cxf* ga = (const cxf*)GA;
        cxf* gb = (cxf*)GB;
        switch (knr) {
            case 9: k_requad_theta_dense<9><<<g, 128, smw, st>>>(ra, nseq, rq.theta_w, rq.nra, rq.nrb, ga, gb); break;
            case 17: k_requad_theta_dense<17><<<g, 128, smw, st>>>(ra, nseq, rq.theta_w, rq.nra, rq.nrb, ga, gb); break;
            case 25: k_requad_theta_dense<25><<<g, 128, smw, st>>>(ra, nseq, rq.theta_w, rq.nra, rq.nrb, ga, gb); break;
            default: k_requad_theta_dense<33><<<g, 128, smw, st>>>(ra, nseq, rq.theta_w, rq.nra, rq.nrb, ga, gb); break;
        }
        return;
    }
    k_requad_spec_cols<Tc><<<nblk((int64_t)nbox * R * (ra.big / 2), kWarps), 32 * kWarps, sm, st>>>(ra, nbox, R, GA, GB);
}

// the transposed theta pass (GB -> GA): the dense form for float32 short circles, else the
// warp-FFT form
template <typename Tc>
void launch_theta_t(const Requad& rq, const RequadArgs& ra, int nbox, int R, const cx<Tc>* GB, cx<Tc>* GA,
                    size_t sm, cudaStream_t st) {
    if (std::is_same<Tc, float>::value && rq.theta_wt) {
        const int64_t nseq = (int64_t)nbox * R;
        const int64_t work = nseq * ra.big;
        const unsigned g = (unsigned)std::min<int64_t>((work + 127) / 128, 152 * 32);
        const int nin = rq.nrb, nout = rq.nra;
        const int knr = nin <= 9 ? 9 : (nin <= 17 ? 17 : (nin <= 25 ? 25 : 33));
        const size_t smw = (size_t)nout * knr * sizeof(float4);
        const cxf* in = (const cxf*)GB;
        cxf* out = (cxf*)GA;
        switch (knr) {
            case 9: k_requad_theta_dense<9><<<g, 128, smw, st>>>(ra, nseq, rq.theta_wt, nin, nout, in, out); break;
            case 17: k_requad_theta_dense<17><<<g, 128, smw, st>>>(ra, nseq, rq.theta_wt, nin, nout, in, out); break;
            case 25: k_requad_theta_dense<25><<<g, 128, smw, st>>>(ra, nseq, rq.theta_wt, nin, nout, in, out); break;
            default: k_requad_theta_dense<33><<<g, 128, smw, st>>>(ra, nseq, rq.theta_wt, nin, nout, in, out); break;
        }
        return;
    }
    k_requad_spec_cols_t<Tc><<<nblk((int64_t)nbox * R * (ra.big / 2), kWarps), 32 * kWarps, sm, st>>>(ra, nbox, R, GB, GA);
}

// Re-quadrature launches.  Tin / Tout: storage types of the input and output levels;
// Tc: compute type, always the parent's (the coarser of the two; precision never decreases
// with depth).  Going up, the parent's signature needs no more.  Going down, the parent's
// data carries only its own precision, so interpolating it in that type adds round-off of
// the size it already has; the child's own part is added in the child's type.
//   M2M l -> l-1, transposed L2L l+1 -> l: level l-1 (resp. l)
//   L2L l -> l+1, transposed M2M l-1 -> l: level l (resp. l-1)
template <typename Tin, typename Tc, typename Tout>
void launch_up(hfmm_plan_s* P, int l, int R, cudaStream_t st) {
    RequadArgs ra = P->up[l].args;
    ra.tw.pool = pool_of<Tc>(P);
    DevLevel& c = P->lev[l];
    DevLevel& p = P->lev[l - 1];
    const size_t sm = (size_t)kWarps * 2 * ra.maxlen * sizeof(cx<Tc>);
    const size_t sm3 = (size_t)kWarps * 3 * ra.maxlen * sizeof(cx<Tc>);   // + per-warp child sum
    cx<Tc>* GA = (cx<Tc>*)P->ga;
    cx<Tc>* GB = (cx<Tc>*)P->gb;
    smem_opt_in(k_requad_spec_a<Tin, Tc, kNoShift>, sm);
    smem_opt_in(k_requad_spec_cols<Tc>, sm);
    smem_opt_in(k_requad_spec_c_m2m<Tc, Tout>, sm3);
    k_requad_spec_a<Tin, Tc, kNoShift><<<nblk((int64_t)c.nbox * R * ra.qa.nrows, kWarps), 32 * kWarps, sm, st>>>(
        ra, c.nbox, R, (const cx<Tin>*)c.M, nullptr, nullptr, nullptr, GA);
    launch_theta<Tc>(P->up[l], ra, c.nbox, R, GA, GB, sm, st);
    k_requad_spec_c_m2m<Tc, Tout><<<nblk((int64_t)p.nbox * R * ra.qb.nrows, kWarps), 32 * kWarps, sm3, st>>>(
        ra, p.nbox, R, p.bv.child_start, p.bv.child_count, c.octant, shift_of<Tc>(p), GB, (cx<Tout>*)p.M);
}

// transposed L2L, child l+1 -> parent l: transpose of the forward L2L (down[l] passes)
template <typename Tin, typename Tc, typename Tout>
void launch_l2l_t(hfmm_plan_s* P, int l, int R, cudaStream_t st) {
    RequadArgs ra = P->down[l].args;
    ra.tw.pool = pool_of<Tc>(P);
    DevLevel& c = P->lev[l + 1];
    DevLevel& p = P->lev[l];
    const size_t sm = (size_t)kWarps * 2 * ra.maxlen * sizeof(cx<Tc>);
    const size_t sm3 = (size_t)kWarps * 3 * ra.maxlen * sizeof(cx<Tc>);
    cx<Tc>* GA = (cx<Tc>*)P->ga;
    cx<Tc>* GB = (cx<Tc>*)P->gb;
    smem_opt_in(k_requad_spec_ct<Tin, Tc, kNoShift>, sm);
    smem_opt_in(k_requad_spec_cols_t<Tc>, sm);
    smem_opt_in(k_requad_spec_at_sum<Tc, Tout>, sm3);
    k_requad_spec_ct<Tin, Tc, kNoShift><<<nblk((int64_t)c.nbox * R * ra.qb.nrows, kWarps), 32 * kWarps, sm, st>>>(
        ra, c.nbox, R, (const cx<Tin>*)c.IL, nullptr, nullptr, nullptr, GB);
    launch_theta_t<Tc>(P->down[l], ra, c.nbox, R, GB, GA, sm, st);
    k_requad_spec_at_sum<Tc, Tout><<<nblk((int64_t)p.nbox * R * ra.qa.nrows, kWarps), 32 * kWarps, sm3, st>>>(
        ra, p.nbox, R, p.bv.child_start, p.bv.child_count, c.octant, shift_of<Tc>(p), GA, (cx<Tout>*)p.IL);
}

template <typename Tin, typename Tc, typename Tout>
void launch_down(hfmm_plan_s* P, int l, int R, cudaStream_t st) {
    RequadArgs ra = P->down[l].args;
    ra.tw.pool = pool_of<Tc>(P);
    DevLevel& p = P->lev[l];
    DevLevel& c = P->lev[l + 1];
    const size_t sm = (size_t)kWarps * 2 * ra.maxlen * sizeof(cx<Tc>);
    cx<Tc>* GA = (cx<Tc>*)P->ga;
    cx<Tc>* GB = (cx<Tc>*)P->gb;
    smem_opt_in(k_requad_spec_a<Tin, Tc, kShiftConj>, sm);
    smem_opt_in(k_requad_spec_cols<Tc>, sm);
    smem_opt_in(k_requad_spec_c_l2l<Tc, Tout>, sm);
    k_requad_spec_a<Tin, Tc, kShiftConj><<<nblk((int64_t)c.nbox * R * ra.qa.nrows, kWarps), 32 * kWarps, sm, st>>>(
        ra, c.nbox, R, (const cx<Tin>*)p.IL, c.bv.parent, c.octant, shift_of<Tc>(p), GA);
    launch_theta<Tc>(P->down[l], ra, c.nbox, R, GA, GB, sm, st);
    k_requad_spec_c_l2l<Tc, Tout><<<nblk((int64_t)c.nbox * R * ra.qb.nrows, kWarps), 32 * kWarps, sm, st>>>(
        ra, c.nbox, R, GB, (cx<Tout>*)c.IL);
}

// transposed M2M, parent l-1 -> child l: transpose of the forward M2M (up[l] passes)
template <typename Tin, typename Tc, typename Tout>
void launch_m2m_t(hfmm_plan_s* P, int l, int R, cudaStream_t st) {
    RequadArgs ra = P->up[l].args;
    ra.tw.pool = pool_of<Tc>(P);
    DevLevel& p = P->lev[l - 1];
    DevLevel& c = P->lev[l];
    const size_t sm = (size_t)kWarps * 2 * ra.maxlen * sizeof(cx<Tc>);
    cx<Tc>* GA = (cx<Tc>*)P->ga;
    cx<Tc>* GB = (cx<Tc>*)P->gb;
    smem_opt_in(k_requad_spec_ct<Tin, Tc, kShiftPlain>, sm);
    smem_opt_in(k_requad_spec_cols_t<Tc>, sm);
    smem_opt_in(k_requad_spec_at_add<Tc, Tout>, sm);
    k_requad_spec_ct<Tin, Tc, kShiftPlain><<<nblk((int64_t)c.nbox * R * ra.qb.nrows, kWarps), 32 * kWarps, sm, st>>>(
        ra, c.nbox, R, (const cx<Tin>*)p.M, c.bv.parent, c.octant, shift_of<Tc>(p), GB);
    launch_theta_t<Tc>(P->up[l], ra, c.nbox, R, GB, GA, sm, st);
    k_requad_spec_at_add<Tc, Tout><<<nblk((int64_t)c.nbox * R * ra.qa.nrows, kWarps), 32 * kWarps, sm, st>>>(
        ra, c.nbox, R, GA, (cx<Tout>*)c.M);
}

template <typename S, typename C>
void launch_m2l(hfmm_plan_s* P, int l, int R, cudaStream_t st, bool transposed) {
    DevLevel& d = P->lev[l];
    const cx<S>* in = (const cx<S>*)(transposed ? d.IL : d.M);
    cx<S>* out = (cx<S>*)(transposed ? d.M : d.IL);
    if (!d.m2l_sib) {
        const dim3 g(d.nbox, nblk(d.K, 128));
        const int32_t* es = transposed ? d.islot_t : d.islot;
        if (R == 1)
            k_m2l_box<S, C, 1><<<g, 128, 0, st>>>(d.K, d.ioff, d.iidx, es, (const cx<S>*)d.table, in, R, out);
        else
            k_m2l_box<S, C, 2><<<g, 128, 0, st>>>(d.K, d.ioff, d.iidx, es, (const cx<S>*)d.table, in, R, out);
        return;
    }
    const dim3 g(d.npar, nblk(d.K, 128));
    const int32_t* ps = transposed ? d.pslot_t : d.pslot;
    if (d.npar == 0) return;
    if (R == 1)
        k_m2l_sib<S, C, 1><<<g, 128, 0, st>>>(d.K, d.pfirst, d.pnch, d.poff, d.pu, d.pmask, ps,
                                              (const cx<S>*)d.table, in, R, out);
    else
        k_m2l_sib<S, C, 2><<<g, 128, 0, st>>>(d.K, d.pfirst, d.pnch, d.poff, d.pu, d.pmask, ps,
                                              (const cx<S>*)d.table, in, R, out);
}

// symmetric float32 near field; `variant` selects the register budget (resident blocks per SM)
void launch_sym(int variant, int nunits, const int2* units, const int32_t* start, const int32_t* count,
                const int32_t* noff, const int32_t* nidx, const P2PMixedArgs& a, const cxd* q, cxd* phi,
                cudaStream_t st) {
    const unsigned g = nblk(nunits, 4);
    switch (variant) {
        case 5: k_p2p_mixed_sym_warp<5><<<g, 128, 0, st>>>(units, nunits, start, count, noff, nidx, a, q, phi); break;
        case 6: k_p2p_mixed_sym_warp<6><<<g, 128, 0, st>>>(units, nunits, start, count, noff, nidx, a, q, phi); break;
        case 8: k_p2p_mixed_sym_warp<8><<<g, 128, 0, st>>>(units, nunits, start, count, noff, nidx, a, q, phi); break;
        default: k_p2p_mixed_sym_warp<7><<<g, 128, 0, st>>>(units, nunits, start, count, noff, nidx, a, q, phi); break;
    }
}

void run_m2l(hfmm_plan_s* P, int l, int R, cudaStream_t st, bool transposed);

// Kernel tuner for M2L: time the per-box and the sibling-group kernels on each level (the
// plan's own lists and tables, the apply's workspace, max_rhs right-hand sides; one warm-up
// and one timed launch each) and keep the faster.  Both give the same result.
hfmm_status tune_m2l(hfmm_plan_s* P) {
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int l = 2; l <= P->hp.lf; ++l) {
        float t[2] = {0.f, 0.f};
        for (int v = 0; v < 2; ++v) {
            P->lev[l].m2l_sib = v == 1;
            run_m2l(P, l, P->rmax, 0, false);
            CK(cudaEventRecord(e0, 0));
            run_m2l(P, l, P->rmax, 0, false);
            CK(cudaEventRecord(e1, 0));
            CK(cudaEventSynchronize(e1));
            CK(cudaEventElapsedTime(&t[v], e0, e1));
        }
        P->lev[l].m2l_sib = t[1] < t[0];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaGetLastError());
    return HFMM_OK;
}

// Kernel tuner: time each register budget of the symmetric near field on the plan's own units
// (two launches each into the plan's workspace, after one warm-up) and keep the fastest.
hfmm_status tune_sym_variant(hfmm_plan_s* P) {
    if (!(P->sym && P->near_prec == kFP32) || P->nsymunits == 0) return HFMM_OK;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaMemset(P->qs, 0, sizeof(cxd) * (size_t)P->hp.ns));
    float best = -1.f;
    for (int v : {5, 6, 7, 8}) {
        launch_sym(v, P->nsymunits, P->symunits, P->tstart, P->tcount, P->noff, P->nidx, P->mixed, P->qs, P->phis, 0);
        CK(cudaEventRecord(e0, 0));
        for (int i = 0; i < 2; ++i)
            launch_sym(v, P->nsymunits, P->symunits, P->tstart, P->tcount, P->noff, P->nidx, P->mixed, P->qs,
                       P->phis, 0);
        CK(cudaEventRecord(e1, 0));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (best < 0.f || ms < best) {
            best = ms;
            P->sym_variant = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaGetLastError());
    return HFMM_OK;
}

// type codes of a level's signatures and arithmetic: 0 float, 1 double, 2 double-float
// (float64 levels of the mixed policy store and compute in double-float pairs)
int store_code(hfmm_plan_s* P, int l) {
    const int p = P->lev[l].prec;
    return p == kFP32 ? 0 : (p == kDF ? 2 : 1);
}
int compute_code(hfmm_plan_s* P, int l) { return store_code(P, l); }

template <typename Fn>
bool dispatch3(int sin, int cc, int sout, Fn fn) {
    // precision only grows with depth (float32 < double-float < float64); cc is the parent's
    if (sin == 1 && cc == 1 && sout == 1) fn(double{}, double{}, double{});
    else if (sin == 2 && cc == 2 && sout == 2) fn(df{}, df{}, df{});
    else if (sin == 0 && cc == 0 && sout == 0) fn(float{}, float{}, float{});
    // up: child (finer type) -> parent
    else if (sin == 2 && cc == 0 && sout == 0) fn(df{}, float{}, float{});
    else if (sin == 1 && cc == 2 && sout == 2) fn(double{}, df{}, df{});
    else if (sin == 1 && cc == 0 && sout == 0) fn(double{}, float{}, float{});
    // down: parent -> child (finer type)
    else if (sin == 0 && cc == 0 && sout == 2) fn(float{}, float{}, df{});
    else if (sin == 0 && cc == 0 && sout == 1) fn(float{}, float{}, double{});
    else if (sin == 2 && cc == 2 && sout == 1) fn(df{}, df{}, double{});
    else return false;
    return true;
}

void run_up(hfmm_plan_s* P, int l, int R, cudaStream_t st) {
    dispatch3(store_code(P, l), compute_code(P, l - 1), store_code(P, l - 1), [&](auto a, auto b, auto c) {
        launch_up<decltype(a), decltype(b), decltype(c)>(P, l, R, st);
    });
}
void run_down(hfmm_plan_s* P, int l, int R, cudaStream_t st) {
    dispatch3(store_code(P, l), compute_code(P, l), store_code(P, l + 1), [&](auto a, auto b, auto c) {
        launch_down<decltype(a), decltype(b), decltype(c)>(P, l, R, st);
    });
}
void run_l2l_t(hfmm_plan_s* P, int l, int R, cudaStream_t st) {
    dispatch3(store_code(P, l + 1), compute_code(P, l), store_code(P, l), [&](auto a, auto b, auto c) {
        launch_l2l_t<decltype(a), decltype(b), decltype(c)>(P, l, R, st);
    });
}
void run_m2m_t(hfmm_plan_s* P, int l, int R, cudaStream_t st) {
    dispatch3(store_code(P, l - 1), compute_code(P, l - 1), store_code(P, l), [&](auto a, auto b, auto c) {
        launch_m2m_t<decltype(a), decltype(b), decltype(c)>(P, l, R, st);
    });
}
void run_m2l(hfmm_plan_s* P, int l, int R, cudaStream_t st, bool transposed) {
    const int cc = compute_code(P, l);
    if (cc == 0) launch_m2l<float, float>(P, l, R, st, transposed);
    else if (cc == 1) launch_m2l<double, double>(P, l, R, st, transposed);
    else launch_m2l<df, df>(P, l, R, st, transposed);
}

// double-float levels evaluate their plane waves in double-float
bool use_df(hfmm_plan_s* P, int l) { return P->lev[l].prec == kDF; }

// points -> signature at the leaves of level l: S2M (sources, sign +1) or transposed L2T
// (targets, sign -1, weighted); other boxes of the level are left as they are
template <typename T>
void launch_s2m(hfmm_plan_s* P, int l, int R, cudaStream_t st, bool transposed = false) {
    DevLevel& d = P->lev[l];
    if (d.nleaf == 0) return;
    const int32_t* start = transposed ? d.tstart : d.sstart;
    const int32_t* count = transposed ? d.tcount : d.scount;
    const double* px = transposed ? P->tx : P->sx;
    const double* py = transposed ? P->ty : P->sy;
    const double* pz = transposed ? P->tz : P->sz;
    const cxd* charges = transposed ? P->phis : P->qs;
    void* out = transposed ? d.IL : d.M;
    const double sign = transposed ? -1.0 : 1.0;
    const double* wk = transposed ? d.qv.w : nullptr;
    const double kt = P->hp.kappa / (2.0 * 3.14159265358979323846);
    BoxView bl = d.bv;
    bl.leaf = d.leaf;
    dim3 grid(d.nleaf, nblk(d.qv.npair, kS2MThreads));
    if (std::is_same<T, double>::value && P->tab_s) {
        // float64 leaf with plane-wave tables (uniform trees): S2M reads the sources' table as
        // stored, the transposed L2T the targets' table conjugated
        const cxd* E = transposed ? P->tab_t : P->tab_s;
        const dim3 g(d.nbox, nblk(d.qv.npair, kTabThreads));
        if (transposed) {
            if (R == 1) k_s2m_tab<1, true><<<g, kTabThreads, 0, st>>>(d.qv, start, count, E, charges, R, (cxd*)out, wk);
            else k_s2m_tab<4, true><<<g, kTabThreads, 0, st>>>(d.qv, start, count, E, charges, R, (cxd*)out, wk);
        } else {
            if (R == 1) k_s2m_tab<1, false><<<g, kTabThreads, 0, st>>>(d.qv, start, count, E, charges, R, (cxd*)out, wk);
            else k_s2m_tab<4, false><<<g, kTabThreads, 0, st>>>(d.qv, start, count, E, charges, R, (cxd*)out, wk);
        }
        return;
    }
    if (std::is_same<T, double>::value && use_df(P, l)) {
        if (R == 1)
            k_s2m_df<1><<<grid, kS2MThreads, 0, st>>>(bl, d.qv, start, count, px, py, pz, charges, R, kt,
                                                      P->cis_tab, (cx<df>*)out, sign, wk);
        else
            k_s2m_df<4><<<grid, kS2MThreads, 0, st>>>(bl, d.qv, start, count, px, py, pz, charges, R, kt,
                                                      P->cis_tab, (cx<df>*)out, sign, wk);
        return;
    }
    if (R == 1)
        k_s2m<T, 1><<<grid, kS2MThreads, 0, st>>>(bl, d.qv, start, count, px, py, pz, charges, R, kt,
                                                  (cx<T>*)out, sign, wk);
    else if (std::is_same<T, float>::value && R >= 16)
        k_s2m<float, 16><<<grid, kS2MThreads, 0, st>>>(bl, d.qv, start, count, px, py, pz, charges, R, kt,
                                                       (cxf*)out, sign, wk);
    else
        k_s2m<T, 4><<<grid, kS2MThreads, 0, st>>>(bl, d.qv, start, count, px, py, pz, charges, R, kt,
                                                  (cx<T>*)out, sign, wk);
}

// signature -> points at the leaves of level l: L2T (targets, sign +1, weighted) or
// transposed S2M (sources, sign -1); adds to the points' values
template <typename T>
void launch_l2t(hfmm_plan_s* P, int l, int R, cudaStream_t st, bool transposed = false) {
    DevLevel& d = P->lev[l];
    if (d.nleaf == 0) return;
    const int32_t* start = transposed ? d.sstart : d.tstart;
    const int32_t* count = transposed ? d.scount : d.tcount;
    const double* px = transposed ? P->sx : P->tx;
    const double* py = transposed ? P->sy : P->ty;
    const double* pz = transposed ? P->sz : P->tz;
    const void* in = transposed ? d.M : d.IL;
    cxd* out = transposed ? P->qs : P->phis;
    const double sign = transposed ? -1.0 : 1.0;
    const double* wk = transposed ? nullptr : d.qv.w;
    const double kt = P->hp.kappa / (2.0 * 3.14159265358979323846);
    BoxView bl = d.bv;
    bl.leaf = d.leaf;
    const dim3 grid(d.nleaf, nblk(transposed ? d.max_src : d.max_tgt, kL2TThreads));
    const int2* units = transposed ? d.sunits : d.tunits;
    const int nu = transposed ? d.nsunits : d.ntunits;
    if (std::is_same<T, double>::value && P->tab_s) {
        // float64 leaf with plane-wave tables (uniform trees): L2T reads the targets' table
        // conjugated, the transposed S2M the sources' table as stored
        const cxd* E = transposed ? P->tab_s : P->tab_t;
        if (nu > 0) {
            const unsigned th = 32 * kL2TabWarps;
            const cxd* Lin = (const cxd*)in;
            if (transposed) {
                if (R == 1) k_l2t_tab<1, false><<<nu, th, 0, st>>>(units, d.qv, start, count, E, Lin, R, out, wk);
                else k_l2t_tab<4, false><<<nu, th, 0, st>>>(units, d.qv, start, count, E, Lin, R, out, wk);
            } else {
                if (R == 1) k_l2t_tab<1, true><<<nu, th, 0, st>>>(units, d.qv, start, count, E, Lin, R, out, wk);
                else k_l2t_tab<4, true><<<nu, th, 0, st>>>(units, d.qv, start, count, E, Lin, R, out, wk);
            }
        }
        return;
    }
    if (std::is_same<T, double>::value && use_df(P, l)) {
        if (nu > 0) {
            if (R == 1)
                k_l2t_df_warp<1><<<nblk(nu, 4), 128, 0, st>>>(units, nu, d.bv, d.qv, d.sdf, start, count, px, py, pz,
                                                             (const cx<df>*)in, R, P->cis_tab, out, sign, wk);
            else
                k_l2t_df_warp<4><<<nblk(nu, 4), 128, 0, st>>>(units, nu, d.bv, d.qv, d.sdf, start, count, px, py, pz,
                                                             (const cx<df>*)in, R, P->cis_tab, out, sign, wk);
        }
        return;
    }
    if (R == 1)
        k_l2t<T, 1><<<grid, kL2TThreads, 0, st>>>(bl, d.qv, start, count, px, py, pz, (const cx<T>*)in, R, kt,
                                                  out, sign, wk);
    else if (std::is_same<T, float>::value && R >= 16)
        k_l2t<float, 16><<<grid, kL2TThreads, 0, st>>>(bl, d.qv, start, count, px, py, pz, (const cxf*)in, R, kt,
                                                       out, sign, wk);
    else
        k_l2t<T, 4><<<grid, kL2TThreads, 0, st>>>(bl, d.qv, start, count, px, py, pz, (const cx<T>*)in, R, kt,
                                                  out, sign, wk);
}

// S2M / L2T of every level that has leaves (a uniform tree: the leaf level only)
void run_s2m(hfmm_plan_s* P, int l, int R, cudaStream_t st, bool transposed = false) {
    if (P->lev[l].prec == kFP32) launch_s2m<float>(P, l, R, st, transposed);
    else launch_s2m<double>(P, l, R, st, transposed);
}
void run_l2t(hfmm_plan_s* P, int l, int R, cudaStream_t st, bool transposed = false) {
    if (P->lev[l].prec == kFP32) launch_l2t<float>(P, l, R, st, transposed);
    else launch_l2t<double>(P, l, R, st, transposed);
}

// transposed far field up to (not including) the transposed S2M: conj(w) on the targets
// (P->phis) -> Lambda_M at the leaf level (M buffers); marks stages 3..6
template <typename Mark>
void transposed_far_chain(hfmm_plan_s* P, int R, cudaStream_t st, Mark mark) {
    const int lf = P->hp.lf;
    // transposed L2T: weighted plane-wave sums of the targets into Lambda_L at the leaves
    run_s2m(P, lf, R, st, true);
    mark(3);
    // transposed L2L, leaf level up to level 2 (it writes every parent; the leaves of an
    // adaptive tree's coarser levels then take their transposed L2T)
    for (int l = lf - 1; l >= 2; --l) {
        run_l2l_t(P, l, R, st);
        run_s2m(P, l, R, st, true);
    }
    mark(4);
    // transposed M2L: the opposite transfer vectors
    for (int l = 2; l <= lf; ++l) run_m2l(P, l, R, st, true);
    mark(5);
    // transposed M2M, level 2 down to the leaf level, added to the M2L part
    for (int l = 3; l <= lf; ++l) run_m2m_t(P, l, R, st);
    mark(6);
}

hfmm_status check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HFMM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return HFMM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void hfmm_default_options(hfmm_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->alpha_ladder[0] = 0.8;
    opt->alpha_ladder[1] = 0.6;
    opt->alpha_ladder[2] = 0.0;
    opt->alpha_ladder[3] = 0.0;
    opt->eps_scale = 0.25;
    opt->max_leaf = 64;
    opt->depth = 0;
    opt->has_root = 0;
    opt->root[3] = 1.0;
    opt->precision = HFMM_PREC_FP64;
    opt->max_rhs = 1;
    opt->device = 0;
    opt->flags = 0;
    opt->leaf_table_bytes = -1;
    opt->buffer = 1;
}

const char* hfmm_last_error(void) { return g_err.c_str(); }

hfmm_status hfmm_debug_fail_host_alloc(int after) {
    g_fail_alloc_after = after < 0 ? -1 : after;
    return HFMM_OK;
}

hfmm_status hfmm_plan(const double* sources, int64_t ns, const double* targets, int64_t nt, double kappa,
                      double eps, const hfmm_options* opt_in, hfmm_plan_t* out) {
    g_err.clear();
    if (!out) return fail(HFMM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!sources || !targets || ns < 1 || nt < 1) return fail(HFMM_ERR_ARG, "need ns >= 1, nt >= 1 and non-NULL points");
    if (ns > INT32_MAX || nt > INT32_MAX) return fail(HFMM_ERR_ARG, "ns and nt must fit in int32");
    if (!(kappa > 0.0) || !std::isfinite(kappa)) return fail(HFMM_ERR_ARG, "kappa must be finite and > 0");
    if (!(eps > 0.0 && eps <= 0.1)) return fail(HFMM_ERR_ARG, "eps must be in (0, 0.1]");
    hfmm_options opt;
    hfmm_default_options(&opt);
    if (opt_in) opt = *opt_in;
    if (opt.max_rhs < 1 || opt.max_rhs > 4096) return fail(HFMM_ERR_ARG, "max_rhs must be in [1, 4096]");
    if (opt.max_leaf < 1) return fail(HFMM_ERR_ARG, "max_leaf must be >= 1");
    if (opt.depth < 0 || opt.depth > kTreeBits) return fail(HFMM_ERR_ARG, "depth must be in [0, 20]");
    if (!(opt.eps_scale > 0.0 && opt.eps_scale <= 1.0)) return fail(HFMM_ERR_ARG, "eps_scale must be in (0, 1]");
    if (opt.precision != HFMM_PREC_FP64 && opt.precision != HFMM_PREC_MIXED)
        return fail(HFMM_ERR_ARG, "unknown precision policy");
    if (opt.flags & ~(HFMM_FLAG_REQUIRE_FAR | HFMM_FLAG_HOST_TABLES | HFMM_FLAG_ADAPTIVE))
        return fail(HFMM_ERR_ARG, "unknown flag bits");
    if (opt.leaf_table_bytes < -1) return fail(HFMM_ERR_ARG, "leaf_table_bytes must be -1, 0 or positive");
    if (opt.buffer < 0 || opt.buffer > 2) return fail(HFMM_ERR_ARG, "buffer must be 0 (chosen by the plan), 1 or 2");
    std::vector<double> alphas;
    // default ladder: (0.8, 0.6), or (0.9, 0.8) below eps = 1e-7, where the few terms that
    // l(0.8) keeps beyond k|r| of a corner pair no longer reach eps
    if (opt.alpha_ladder[0] == 0.8 && opt.alpha_ladder[1] == 0.6 && opt.alpha_ladder[2] == 0.0 && eps < 1e-7) {
        opt.alpha_ladder[0] = 0.9;
        opt.alpha_ladder[1] = 0.8;
    }
    for (int i = 0; i < 4 && opt.alpha_ladder[i] != 0.0; ++i) {
        if (!(opt.alpha_ladder[i] >= 0.5 && opt.alpha_ladder[i] <= 1.0))
            return fail(HFMM_ERR_ARG, "alpha values must lie in [0.5, 1]");
        alphas.push_back(opt.alpha_ladder[i]);
    }
    if (alphas.empty()) return fail(HFMM_ERR_ARG, "alpha_ladder is empty");
    for (int64_t i = 0; i < 3 * ns; ++i)
        if (!std::isfinite(sources[i])) return fail(HFMM_ERR_ARG, "non-finite source coordinate");
    for (int64_t i = 0; i < 3 * nt; ++i)
        if (!std::isfinite(targets[i])) return fail(HFMM_ERR_ARG, "non-finite target coordinate");
    if (opt.has_root) {
        if (!(opt.root[3] > 0.0)) return fail(HFMM_ERR_ARG, "root side must be > 0");
        for (int64_t i = 0; i < ns; ++i)
            for (int k = 0; k < 3; ++k)
                if (sources[3 * i + k] < opt.root[k] || sources[3 * i + k] > opt.root[k] + opt.root[3])
                    return fail(HFMM_ERR_ARG, "a source lies outside the given root cube");
        for (int64_t i = 0; i < nt; ++i)
            for (int k = 0; k < 3; ++k)
                if (targets[3 * i + k] < opt.root[k] || targets[3 * i + k] > opt.root[k] + opt.root[3])
                    return fail(HFMM_ERR_ARG, "a target lies outside the given root cube");
    }
    hfmm_plan_s* P = new (std::nothrow) hfmm_plan_s();
    if (!P) return fail(HFMM_ERR_NOMEM, "host allocation failed");
    HostPlan& hp = P->hp;
    try {
        hp.src.assign(sources, sources + 3 * ns);
        hp.tgt.assign(targets, targets + 3 * nt);
        hp.ns = ns;
        hp.nt = nt;
        hp.kappa = kappa;
        hp.eps = eps;
        hp.eps_scale = opt.eps_scale;
        hp.alphas = alphas;
        hp.max_leaf = opt.max_leaf;
        hp.depth_req = opt.depth;
        hp.precision = opt.precision;
        hp.buffer = opt.buffer;
        // inputs of the plan-shape tuner (buffer = 0)
        hp.model_rhs = opt.max_rhs;
        hp.model_near = opt.precision == HFMM_PREC_MIXED ? (eps >= 1e-6 ? kFP32 : (eps >= 1e-11 ? kDF : kFP64)) : kFP64;
        hp.model_sym = ns == nt && (sources == targets || std::memcmp(sources, targets, sizeof(double) * 3 * ns) == 0);
        hp.adaptive = (opt.flags & HFMM_FLAG_ADAPTIVE) ? 1 : 0;
        // adaptive trees evaluate plane waves per leaf level: no float64 leaf tables
        hp.model_table_bytes = hp.adaptive ? 0 : opt.leaf_table_bytes;
        // transfer tables on the device unless asked for on the host (or no device)
        hp.host_tables = opt.device < 0 || (opt.flags & HFMM_FLAG_HOST_TABLES);
        hp.has_root = opt.has_root;
        for (int k = 0; k < 4; ++k) hp.root[k] = opt.root[k];
        std::string e = build_host_plan(hp);
        if (!e.empty()) {
            delete P;
            return fail(HFMM_ERR_ARG, e);
        }
    } catch (const std::bad_alloc&) {
        delete P;
        return fail(HFMM_ERR_NOMEM, "host allocation failed while planning");
    } catch (const std::exception& ex) {
        delete P;
        return fail(HFMM_ERR_ARG, ex.what());
    }
    // FFT lengths are bounded by the warp transforms' shared buffers and index arithmetic
    for (int l = 2; l <= hp.lf; ++l) {
        if (hp.lp[l].quad.ntheta > 1024) {
            delete P;
            return fail(HFMM_ERR_ARG, "N_theta above 1024 is not supported");
        }
        for (int v : hp.lp[l].quad.nphi)
            if (v > 1024) {
                delete P;
                return fail(HFMM_ERR_ARG, "N_phi above 1024 is not supported");
            }
    }
    if ((opt.flags & HFMM_FLAG_REQUIRE_FAR) && hp.lf < 2) {
        std::string why;
        if (hp.occ_depth < 2)
            why = "the occupancy depth is " + std::to_string(hp.occ_depth) + " (fewer than 2 levels)";
        else if (kappa * hp.side / 4.0 < 6.0)
            why = "level 2 boxes are below a wavelength (kappa a_2 = " + std::to_string(kappa * hp.side / 4.0) + " < 6)";
        else
            why = "the round-off rule rejects level 2 for every alpha in every allowed precision";
        delete P;
        return fail(HFMM_ERR_UNSTABLE, "no far-field level: " + why);
    }
    P->rmax = opt.max_rhs;
    P->device = opt.device;
    P->tab_budget = hp.adaptive ? 0 : opt.leaf_table_bytes;
    if (opt.precision == HFMM_PREC_MIXED) P->near_prec = eps >= 1e-6 ? kFP32 : (eps >= 1e-11 ? kDF : kFP64);
    P->sym = ns == nt && (sources == targets || std::memcmp(sources, targets, sizeof(double) * 3 * ns) == 0) &&
             P->hp.src_perm == P->hp.tgt_perm && P->hp.src_count == P->hp.tgt_count;
    if (opt.device >= 0) {
        hfmm_status s = upload_plan(P);
        if (s == HFMM_OK) s = tune_sym_variant(P);
        if (s == HFMM_OK) s = tune_m2l(P);
        if (s != HFMM_OK) {
            std::string msg = g_err;
            hfmm_destroy(P);
            return fail(s, msg);
        }
    }
    *out = P;
    return HFMM_OK;
}

hfmm_status hfmm_destroy(hfmm_plan_t P) {
    if (!P) return HFMM_OK;
    if (P->device >= 0) {
        cudaSetDevice(P->device);
        for (void* v : P->allocs) cudaFree(v);
        for (int i = 0; i <= HFMM_N_STAGES; ++i)
            if (P->ev[i]) cudaEventDestroy(P->ev[i]);
    }
    delete P;
    return HFMM_OK;
}

hfmm_status hfmm_set_timing(hfmm_plan_t P, int on) {
    if (!P) return fail(HFMM_ERR_ARG, "plan is NULL");
    if (P->device < 0) return fail(HFMM_ERR_STATE, "host-only plan");
    P->timing = on != 0;
    P->ev_recorded = false;
    return HFMM_OK;
}

hfmm_status hfmm_apply(hfmm_plan_t P, const void* q, void* phi, int nrhs, hfmm_dtype dtype, void* stream) {
    if (!P) return fail(HFMM_ERR_ARG, "plan is NULL");
    if (P->device < 0) return fail(HFMM_ERR_STATE, "host-only plan has no device data");
    if (!q || !phi) return fail(HFMM_ERR_ARG, "q and phi must be device pointers");
    if (nrhs < 1 || nrhs > P->rmax) return fail(HFMM_ERR_ARG, "nrhs must be in [1, max_rhs]");
    if (dtype != HFMM_C64 && dtype != HFMM_C128) return fail(HFMM_ERR_ARG, "unknown dtype");
    CK(cudaSetDevice(P->device));
    cudaStream_t st = (cudaStream_t)stream;
    HostPlan& hp = P->hp;
    const int R = nrhs;
    const int lf = hp.lf;
    auto mark = [&](int i) {
        if (P->timing) cudaEventRecord(P->ev[i], st);
    };
    mark(0);
    if (dtype == HFMM_C64)
        k_permute_in<float, false><<<nblk(hp.ns * R, 256), 256, 0, st>>>((const cxf*)q, hp.ns, R, P->src_perm, P->qs);
    else
        k_permute_in<double, false><<<nblk(hp.ns * R, 256), 256, 0, st>>>((const cxd*)q, hp.ns, R, P->src_perm, P->qs);
    mark(1);
    const int nleaf = (int)hp.leaf_level.size();
    const dim3 g_fwd(nleaf, nblk(P->max_tgt_leaf, kP2PThreads));
    const df kt_df = df_from_double(hp.kappa / (2.0 * 3.14159265358979323846));
    if (P->near_prec == kFP32 && P->sym && R == 1) {
        CK(cudaMemsetAsync(P->phis, 0, sizeof(cxd) * (size_t)hp.nt, st));
        if (P->nsymunits > 0)
            launch_sym(P->sym_variant, P->nsymunits, P->symunits, P->tstart, P->tcount, P->noff, P->nidx, P->mixed,
                       P->qs, P->phis, st);
    } else if (P->near_prec == kFP32 && R >= hfmm_plan_s::kTc5MinRhs) {
        launch_t5(P, false, R, st);
    } else if (P->near_prec == kFP32 && R >= hfmm_plan_s::kTcMinRhs) {
        // static + dynamic shared memory exceeds 48 KiB: opt in explicitly
        cudaFuncSetAttribute(k_p2p_mixed_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcDynSmem);
        if (P->ntunits64 > 0)
            k_p2p_mixed_tc<<<P->ntunits64, 128, kTcDynSmem, st>>>(P->tunits64, P->ntunits64, P->tstart, P->tcount,
                                                                P->sstart, P->scount, P->noff, P->nidx, P->mixed,
                                                                P->qs, P->phis, R);
    } else if (P->near_prec == kFP32) {
        if (P->ntunits > 0) {
            if (R == 1)
                k_p2p_mixed_warp<1><<<nblk(P->ntunits, 4), 128, 0, st>>>(P->tunits, P->ntunits, P->tstart, P->tcount,
                                                                         P->sstart, P->scount, P->noff, P->nidx,
                                                                         P->mixed, P->qs, P->phis, R);
            else
                k_p2p_mixed_warp<4><<<nblk(P->ntunits, 4), 128, 0, st>>>(P->tunits, P->ntunits, P->tstart, P->tcount,
                                                                         P->sstart, P->scount, P->noff, P->nidx,
                                                                         P->mixed, P->qs, P->phis, R);
        }
    } else if (P->near_prec == kDF) {
        if (P->ntunits > 0) {
            if (R == 1)
                k_p2p_df_warp<1><<<nblk(P->ntunits, 4), 128, 0, st>>>(P->tunits, P->ntunits, P->tstart, P->tcount,
                                                                      P->sstart, P->scount, P->noff, P->nidx,
                                                                      P->tpos_df, P->spos_df, kt_df, P->cis_tab,
                                                                      P->qs, P->phis, R);
            else
                k_p2p_df_warp<4><<<nblk(P->ntunits, 4), 128, 0, st>>>(P->tunits, P->ntunits, P->tstart, P->tcount,
                                                                      P->sstart, P->scount, P->noff, P->nidx,
                                                                      P->tpos_df, P->spos_df, kt_df, P->cis_tab,
                                                                      P->qs, P->phis, R);
        }
    } else {
        k_p2p_fp64<<<g_fwd, kP2PThreads, 0, st>>>(nleaf, P->tstart, P->tcount, P->sstart, P->scount, P->noff,
                                                  P->nidx, P->tx, P->ty, P->tz, P->sx, P->sy, P->sz, P->qs,
                                                  P->phis, R, hp.kappa);
    }
    mark(2);
    if (lf >= 2) {
        run_s2m(P, lf, R, st);
        mark(3);
        // M2M writes every parent; the leaves of an adaptive tree's coarser levels then take
        // their S2M
        for (int l = lf; l >= 3; --l) {
            run_up(P, l, R, st);
            run_s2m(P, l - 1, R, st);
        }
        mark(4);
        for (int l = 2; l <= lf; ++l) run_m2l(P, l, R, st, false);
        mark(5);
        for (int l = 2; l < lf; ++l) run_down(P, l, R, st);
        mark(6);
        for (int l = 2; l <= lf; ++l) run_l2t(P, l, R, st);
        mark(7);
    } else {
        for (int i = 3; i <= 7; ++i) mark(i);
    }
    if (dtype == HFMM_C64)
        k_permute_out<float, false><<<nblk(hp.nt * R, 256), 256, 0, st>>>(P->phis, hp.nt, R, P->tgt_perm, (cxf*)phi);
    else
        k_permute_out<double, false><<<nblk(hp.nt * R, 256), 256, 0, st>>>(P->phis, hp.nt, R, P->tgt_perm, (cxd*)phi);
    mark(8);
    P->ev_recorded = P->timing;
    return check_launch("hfmm_apply");
}

hfmm_status hfmm_apply_adjoint(hfmm_plan_t P, const void* w, void* out, int nrhs, hfmm_dtype dtype,
                               void* stream) {
    if (!P) return fail(HFMM_ERR_ARG, "plan is NULL");
    if (P->device < 0) return fail(HFMM_ERR_STATE, "host-only plan has no device data");
    if (!w || !out) return fail(HFMM_ERR_ARG, "w and out must be device pointers");
    if (nrhs < 1 || nrhs > P->rmax) return fail(HFMM_ERR_ARG, "nrhs must be in [1, max_rhs]");
    if (dtype != HFMM_C64 && dtype != HFMM_C128) return fail(HFMM_ERR_ARG, "unknown dtype");
    CK(cudaSetDevice(P->device));
    cudaStream_t st = (cudaStream_t)stream;
    HostPlan& hp = P->hp;
    const int R = nrhs;
    const int lf = hp.lf;
    auto mark = [&](int i) {
        if (P->timing) cudaEventRecord(P->ev[i], st);
    };
    mark(0);
    // conj(w) on the targets, sorted, into the target-side buffer
    if (dtype == HFMM_C64)
        k_permute_in<float, true><<<nblk(hp.nt * R, 256), 256, 0, st>>>((const cxf*)w, hp.nt, R, P->tgt_perm, P->phis);
    else
        k_permute_in<double, true><<<nblk(hp.nt * R, 256), 256, 0, st>>>((const cxd*)w, hp.nt, R, P->tgt_perm, P->phis);
    mark(1);
    // transposed near field: source boxes gather the targets of their neighbours
    const int nleaf = (int)hp.leaf_level.size();
    const dim3 g_adj(nleaf, nblk(P->max_src_leaf, kP2PThreads));
    const df kt_df = df_from_double(hp.kappa / (2.0 * 3.14159265358979323846));
    if (P->near_prec == kFP32 && P->sym && R == 1) {
        CK(cudaMemsetAsync(P->qs, 0, sizeof(cxd) * (size_t)hp.ns, st));
        if (P->nsymunits > 0)
            launch_sym(P->sym_variant, P->nsymunits, P->symunits, P->sstart, P->scount, P->noff, P->nidx, P->mixed,
                       P->phis, P->qs, st);
    } else if (P->near_prec == kFP32 && R >= hfmm_plan_s::kTc5MinRhs) {
        launch_t5(P, true, R, st);
    } else if (P->near_prec == kFP32 && R >= hfmm_plan_s::kTcMinRhs) {
        P2PMixedArgs a = P->mixed;
        std::swap(a.tpt, a.spt);
        std::swap(a.tof, a.sof);
        // static + dynamic shared memory exceeds 48 KiB: opt in explicitly
        cudaFuncSetAttribute(k_p2p_mixed_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcDynSmem);
        if (P->nsunits64 > 0)
            k_p2p_mixed_tc<<<P->nsunits64, 128, kTcDynSmem, st>>>(P->sunits64, P->nsunits64, P->sstart, P->scount,
                                                                P->tstart, P->tcount, P->noff, P->nidx, a, P->phis,
                                                                P->qs, R);
    } else if (P->near_prec == kFP32) {
        P2PMixedArgs a = P->mixed;
        std::swap(a.tpt, a.spt);
        std::swap(a.tof, a.sof);
        if (P->nsunits > 0) {
            if (R == 1)
                k_p2p_mixed_warp<1><<<nblk(P->nsunits, 4), 128, 0, st>>>(P->sunits, P->nsunits, P->sstart, P->scount,
                                                                         P->tstart, P->tcount, P->noff, P->nidx, a,
                                                                         P->phis, P->qs, R);
            else
                k_p2p_mixed_warp<4><<<nblk(P->nsunits, 4), 128, 0, st>>>(P->sunits, P->nsunits, P->sstart, P->scount,
                                                                         P->tstart, P->tcount, P->noff, P->nidx, a,
                                                                         P->phis, P->qs, R);
        }
    } else if (P->near_prec == kDF) {
        if (P->nsunits > 0) {
            if (R == 1)
                k_p2p_df_warp<1><<<nblk(P->nsunits, 4), 128, 0, st>>>(P->sunits, P->nsunits, P->sstart, P->scount,
                                                                      P->tstart, P->tcount, P->noff, P->nidx,
                                                                      P->spos_df, P->tpos_df, kt_df, P->cis_tab,
                                                                      P->phis, P->qs, R);
            else
                k_p2p_df_warp<4><<<nblk(P->nsunits, 4), 128, 0, st>>>(P->sunits, P->nsunits, P->sstart, P->scount,
                                                                      P->tstart, P->tcount, P->noff, P->nidx,
                                                                      P->spos_df, P->tpos_df, kt_df, P->cis_tab,
                                                                      P->phis, P->qs, R);
        }
    } else {
        k_p2p_fp64<<<g_adj, kP2PThreads, 0, st>>>(nleaf, P->sstart, P->scount, P->tstart, P->tcount, P->noff,
                                                  P->nidx, P->sx, P->sy, P->sz, P->tx, P->ty, P->tz, P->phis,
                                                  P->qs, R, hp.kappa);
    }
    mark(2);
    if (lf >= 2) {
        transposed_far_chain(P, R, st, mark);
        // transposed S2M: plane-wave sums back onto the sources of every level's leaves
        for (int l = 2; l <= lf; ++l) run_l2t(P, l, R, st, true);
        mark(7);
    } else {
        for (int i = 3; i <= 7; ++i) mark(i);
    }
    if (dtype == HFMM_C64)
        k_permute_out<float, true><<<nblk(hp.ns * R, 256), 256, 0, st>>>(P->qs, hp.ns, R, P->src_perm, (cxf*)out);
    else
        k_permute_out<double, true><<<nblk(hp.ns * R, 256), 256, 0, st>>>(P->qs, hp.ns, R, P->src_perm, (cxd*)out);
    mark(8);
    P->ev_recorded = P->timing;
    return check_launch("hfmm_apply_adjoint");
}

hfmm_status hfmm_grad_sources(hfmm_plan_t P, const void* q, const void* g, double* grad, int nrhs,
                              hfmm_dtype dtype, void* stream) {
    if (!P) return fail(HFMM_ERR_ARG, "plan is NULL");
    if (P->device < 0) return fail(HFMM_ERR_STATE, "host-only plan has no device data");
    if (!q || !g || !grad) return fail(HFMM_ERR_ARG, "q, g and grad must be device pointers");
    if (nrhs < 1 || nrhs > P->rmax) return fail(HFMM_ERR_ARG, "nrhs must be in [1, max_rhs]");
    if (dtype != HFMM_C64 && dtype != HFMM_C128) return fail(HFMM_ERR_ARG, "unknown dtype");
    CK(cudaSetDevice(P->device));
    cudaStream_t st = (cudaStream_t)stream;
    HostPlan& hp = P->hp;
    const int R = nrhs;
    const int lf = hp.lf;
    auto mark = [&](int i) {
        if (P->timing) cudaEventRecord(P->ev[i], st);
    };
    mark(0);
    if (dtype == HFMM_C64) {
        k_permute_in<float, false><<<nblk(hp.ns * R, 256), 256, 0, st>>>((const cxf*)q, hp.ns, R, P->src_perm, P->qs);
        k_permute_in<float, true><<<nblk(hp.nt * R, 256), 256, 0, st>>>((const cxf*)g, hp.nt, R, P->tgt_perm, P->phis);
    } else {
        k_permute_in<double, false><<<nblk(hp.ns * R, 256), 256, 0, st>>>((const cxd*)q, hp.ns, R, P->src_perm, P->qs);
        k_permute_in<double, true><<<nblk(hp.nt * R, 256), 256, 0, st>>>((const cxd*)g, hp.nt, R, P->tgt_perm, P->phis);
    }
    mark(1);
    const int nleaf = (int)hp.leaf_level.size();
    k_grad_near<<<dim3(nleaf, nblk(P->max_src_leaf, kP2PThreads)), kP2PThreads, 0, st>>>(nleaf, P->sstart, P->scount, P->tstart, P->tcount, P->noff, P->nidx,
                                               P->sx, P->sy, P->sz, P->tx, P->ty, P->tz, P->qs, P->phis, R,
                                               hp.kappa, P->gsort);
    mark(2);
    if (lf >= 2) {
        transposed_far_chain(P, R, st, mark);
        for (int l = 2; l <= lf; ++l) {
            DevLevel& d = P->lev[l];
            if (d.nleaf == 0) continue;
            BoxView bl = d.bv;
            bl.leaf = d.leaf;
            const dim3 gg(d.nleaf, nblk(d.max_src, kL2TThreads));
            const int sc = store_code(P, l);
            if (sc == 1)
                k_grad_far<double, double><<<gg, kL2TThreads, 0, st>>>(bl, d.qv, d.sstart, d.scount, P->sx, P->sy,
                                                                       P->sz, (const cxd*)d.M, P->qs, R, hp.kappa,
                                                                       P->gsort);
            else if (sc == 2)
                k_grad_far<df, double><<<gg, kL2TThreads, 0, st>>>(bl, d.qv, d.sstart, d.scount, P->sx, P->sy, P->sz,
                                                                   (const cx<df>*)d.M, P->qs, R, hp.kappa, P->gsort);
            else
                k_grad_far<float, float><<<gg, kL2TThreads, 0, st>>>(bl, d.qv, d.sstart, d.scount, P->sx, P->sy,
                                                                     P->sz, (const cxf*)d.M, P->qs, R, hp.kappa,
                                                                     P->gsort);
        }
        mark(7);
    } else {
        for (int i = 3; i <= 7; ++i) mark(i);
    }
    k_scatter_grad<<<nblk(hp.ns * 3, 256), 256, 0, st>>>(P->gsort, hp.ns, P->src_perm, grad);
    mark(8);
    P->ev_recorded = P->timing;
    return check_launch("hfmm_grad_sources");
}

hfmm_status hfmm_debug_watchdog_probe(hfmm_plan_t P, void* stream) {
    if (!P) return fail(HFMM_ERR_ARG, "plan is NULL");
    if (P->device < 0 || !P->dev_err) return fail(HFMM_ERR_STATE, "host-only plan");
    CK(cudaSetDevice(P->device));
    k_t5_watchdog_probe<<<1, 32, 0, (cudaStream_t)stream>>>(P->dev_err);
    return check_launch("hfmm_debug_watchdog_probe");
}

hfmm_status hfmm_query(hfmm_plan_t P, hfmm_info* info) {
    if (!P || !info) return fail(HFMM_ERR_ARG, "NULL argument");
    if (P->device >= 0 && P->dev_err) {
        // a kernel of an earlier call gave up a bounded wait: report it once
        int flag = 0;
        CK(cudaSetDevice(P->device));
        CK(cudaMemcpy(&flag, P->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (flag) {
            CK(cudaMemset(P->dev_err, 0, sizeof(int)));
            return fail(HFMM_ERR_TIMEOUT, "a kernel gave up a bounded wait (device watchdog); its results are incomplete");
        }
    }
    std::memset(info, 0, sizeof(*info));
    const HostPlan& hp = P->hp;
    info->ns = hp.ns;
    info->nt = hp.nt;
    info->kappa = hp.kappa;
    info->eps = hp.eps;
    info->occupancy_depth = hp.occ_depth;
    info->lf = hp.lf;
    info->p2p_pairs = hp.p2p_pairs;
    for (int l = 0; l <= hp.lf && l < HFMM_MAX_LEVELS; ++l) {
        info->level_nbox[l] = (int)hp.levels[l].nbox();
        if (l >= 2) {
            const LevelPlan& lp = hp.lp[l];
            info->level_ell[l] = lp.quad.ell;
            info->level_ntheta[l] = lp.quad.ntheta;
            info->level_K[l] = lp.quad.K;
            info->level_precision[l] = lp.prec == kFP32 ? HFMM_LEVEL_FP32 : (lp.prec == kDF ? HFMM_LEVEL_DF : HFMM_LEVEL_FP64);
            info->level_alpha[l] = lp.alpha;
            info->level_round_est[l] = lp.est;
            info->level_ilist_total[l] = (int)hp.levels[l].iidx.size();
        }
    }
    info->workspace_bytes = P->workspace;
    info->p2p_self_pairs = hp.p2p_self_pairs;
    info->near_symmetric = (P->sym && P->near_prec == kFP32) ? 1 : 0;
    info->near_precision = P->near_prec == kFP32 ? HFMM_LEVEL_FP32 : (P->near_prec == kDF ? HFMM_LEVEL_DF : HFMM_LEVEL_FP64);
    info->leaf_tables = P->tab_s != nullptr;
    info->buffer = hp.buffer;
    info->tuned = hp.tuned;
    info->near_variant = (P->sym && P->near_prec == kFP32) ? P->sym_variant : 0;
    info->near_mma_tiles = P->near_prec == kFP32 ? P->t5tiles_fwd : 0;
    for (int b = 0; b < 3; ++b)
        for (int l = 0; l < HFMM_MAX_LEVELS; ++l) info->predicted_ms[b][l] = hp.predicted_ms[b][l];
    info->leaf_table_bytes = P->tab_bytes;
    info->adaptive = hp.adaptive;
    info->nleaf = (int64_t)hp.leaf_level.size();
    for (int l = 0; l <= hp.lf && l < HFMM_MAX_LEVELS; ++l) info->level_nleaf[l] = (int)hp.levels[l].leaf_pos.size();
    if (P->ev_recorded) {
        if (cudaEventSynchronize(P->ev[HFMM_N_STAGES]) != cudaSuccess)
            return fail(HFMM_ERR_CUDA, "event synchronize failed");
        for (int i = 0; i < HFMM_N_STAGES; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, P->ev[i], P->ev[i + 1]);
            info->stage_ms[i] = ms;
        }
    }
    return HFMM_OK;
}

}  // extern "C"

struct hfmm_batch_s {
    std::vector<hfmm_plan_t> plans;
    int device = 0;
    static constexpr int kBranches = 8;
    cudaStream_t cap = nullptr;                 // capture origin
    cudaStream_t br[kBranches] = {};            // concurrent branches inside the graph
    cudaEvent_t fork = nullptr, join[kBranches] = {};
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> key_q;
    std::vector<void*> key_phi;
    int key_r = -1, key_dtype = -1;
    bool warmed = false;
};

extern "C" {

hfmm_status hfmm_batch_destroy(hfmm_batch_t B) {
    if (!B) return HFMM_OK;
    cudaSetDevice(B->device);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    for (int i = 0; i < hfmm_batch_s::kBranches; ++i) {
        if (B->br[i]) cudaStreamDestroy(B->br[i]);
        if (B->join[i]) cudaEventDestroy(B->join[i]);
    }
    if (B->fork) cudaEventDestroy(B->fork);
    if (B->cap) cudaStreamDestroy(B->cap);
    for (hfmm_plan_t p : B->plans) hfmm_destroy(p);
    delete B;
    return HFMM_OK;
}

hfmm_status hfmm_plan_batch(int nprob, const hfmm_problem* probs, const hfmm_options* opt, hfmm_batch_t* out) {
    g_err.clear();
    if (!out) return fail(HFMM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nprob < 1 || !probs) return fail(HFMM_ERR_ARG, "need nprob >= 1 and a problem array");
    hfmm_options o;
    hfmm_default_options(&o);
    if (opt) o = *opt;
    if (o.device < 0) return fail(HFMM_ERR_ARG, "a batch needs a device");
    hfmm_batch_s* B = new (std::nothrow) hfmm_batch_s();
    if (!B) return fail(HFMM_ERR_NOMEM, "host allocation failed");
    B->device = o.device;
    for (int p = 0; p < nprob; ++p) {
        hfmm_plan_t h = nullptr;
        hfmm_status s = hfmm_plan(probs[p].sources, probs[p].ns, probs[p].targets, probs[p].nt, probs[p].kappa,
                                  probs[p].eps, &o, &h);
        if (s != HFMM_OK) {
            std::string msg = "problem " + std::to_string(p) + ": " + g_err;
            hfmm_batch_destroy(B);
            return fail(s, msg);
        }
        B->plans.push_back(h);
    }
    cudaSetDevice(B->device);
    bool ok = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; ok && i < hfmm_batch_s::kBranches; ++i)
        ok = cudaStreamCreateWithFlags(&B->br[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&B->join[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        hfmm_batch_destroy(B);
        return fail(HFMM_ERR_CUDA, "stream/event creation failed");
    }
    *out = B;
    return HFMM_OK;
}

hfmm_status hfmm_batch_plan(hfmm_batch_t B, int p, hfmm_plan_t* plan) {
    if (!B || !plan || p < 0 || p >= (int)B->plans.size()) return fail(HFMM_ERR_ARG, "bad batch index");
    *plan = B->plans[p];
    return HFMM_OK;
}

hfmm_status hfmm_apply_batch(hfmm_batch_t B, const void* const* q, void* const* phi, int nrhs, hfmm_dtype dtype,
                             void* stream) {
    if (!B || !q || !phi) return fail(HFMM_ERR_ARG, "NULL argument");
    const int n = (int)B->plans.size();
    for (int p = 0; p < n; ++p) {
        if (!q[p] || !phi[p]) return fail(HFMM_ERR_ARG, "NULL buffer for problem " + std::to_string(p));
        if (nrhs < 1 || nrhs > B->plans[p]->rmax) return fail(HFMM_ERR_ARG, "nrhs must be in [1, max_rhs]");
    }
    if (dtype != HFMM_C64 && dtype != HFMM_C128) return fail(HFMM_ERR_ARG, "unknown dtype");
    CK(cudaSetDevice(B->device));
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<const void*> kq(q, q + n);
    std::vector<void*> kp(phi, phi + n);
    if (!B->exec || kq != B->key_q || kp != B->key_phi || nrhs != B->key_r || (int)dtype != B->key_dtype) {
        if (!B->warmed) {  // load every kernel once outside the capture
            for (int p = 0; p < n; ++p) TRY(hfmm_apply(B->plans[p], q[p], phi[p], nrhs, dtype, stream));
            CK(cudaStreamSynchronize(st));
            B->warmed = true;
        }
        if (B->exec) {
            cudaGraphExecDestroy(B->exec);
            B->exec = nullptr;
        }
        for (int p = 0; p < n; ++p) B->plans[p]->timing = false;
        CK(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeRelaxed));
        CK(cudaEventRecord(B->fork, B->cap));
        for (int i = 0; i < hfmm_batch_s::kBranches; ++i) CK(cudaStreamWaitEvent(B->br[i], B->fork, 0));
        hfmm_status s = HFMM_OK;
        for (int p = 0; p < n && s == HFMM_OK; ++p)
            s = hfmm_apply(B->plans[p], q[p], phi[p], nrhs, dtype, B->br[p % hfmm_batch_s::kBranches]);
        for (int i = 0; i < hfmm_batch_s::kBranches; ++i) {
            cudaEventRecord(B->join[i], B->br[i]);
            cudaStreamWaitEvent(B->cap, B->join[i], 0);
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(B->cap, &graph);
        if (s != HFMM_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (e != cudaSuccess) return fail(HFMM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&B->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            B->exec = nullptr;
            return fail(HFMM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        }
        B->key_q = kq;
        B->key_phi = kp;
        B->key_r = nrhs;
        B->key_dtype = (int)dtype;
    }
    CK(cudaGraphLaunch(B->exec, st));
    return HFMM_OK;
}

int64_t hfmm_debug_get(hfmm_plan_t P, int what, int level, int64_t arg, void* out, int64_t cap) {
    if (!P) return -1;
    const HostPlan& hp = P->hp;
    auto give = [&](const void* src, int64_t count, size_t esz) -> int64_t {
        if (out && count > 0) std::memcpy(out, src, (size_t)std::min(count, cap) * esz);
        return count;
    };
    const bool lev_ok = level >= 0 && level <= hp.lf;
    switch (what) {
        case HFMM_GET_BOX_IDX:
            if (!lev_ok) return -1;
            return give(hp.levels[level].idx.data(), (int64_t)hp.levels[level].idx.size(), 4);
        case HFMM_GET_BOX_PARENT:
            if (!lev_ok) return -1;
            return give(hp.levels[level].parent.data(), (int64_t)hp.levels[level].parent.size(), 4);
        case HFMM_GET_ILIST_OFF:
            if (!lev_ok || level < 2) return -1;
            return give(hp.levels[level].ioff.data(), (int64_t)hp.levels[level].ioff.size(), 4);
        case HFMM_GET_ILIST_IDX:
            if (!lev_ok || level < 2) return -1;
            return give(hp.levels[level].iidx.data(), (int64_t)hp.levels[level].iidx.size(), 4);
        case HFMM_GET_ILIST_V:
            if (!lev_ok || level < 2) return -1;
            return give(hp.levels[level].iv.data(), (int64_t)hp.levels[level].iv.size(), 4);
        case HFMM_GET_NLIST_OFF:
            return give(hp.noff.data(), (int64_t)hp.noff.size(), 4);
        case HFMM_GET_NLIST_IDX:
            return give(hp.nidx.data(), (int64_t)hp.nidx.size(), 4);
        case HFMM_GET_SRC_PERM:
            return give(hp.src_perm.data(), (int64_t)hp.src_perm.size(), 8);
        case HFMM_GET_TGT_PERM:
            return give(hp.tgt_perm.data(), (int64_t)hp.tgt_perm.size(), 8);
        case HFMM_GET_NPHI:
            if (!lev_ok || level < 2) return -1;
            return give(hp.lp[level].quad.nphi.data(), (int64_t)hp.lp[level].quad.nphi.size(), 4);
        case HFMM_GET_TABLE: {
            if (!lev_ok || level < 2 || arg < 0 || arg >= transfer_slots(hp.buffer)) return -1;
            if (!hp.host_tables) {
                // computed on the device: copy the vector's slot back, converted to float64
                const DevLevel& d = P->lev[level];
                bool used = false;
                for (int32_t v : hp.levels[level].iv) used |= (v == arg);
                if (!used || !d.table) return -1;
                const int64_t K = hp.lp[level].quad.K;
                if (out) {
                    const size_t e = d.prec == kFP32 ? sizeof(cxf) : (d.prec == kFP64 ? sizeof(cxd) : sizeof(cx<df>));
                    std::vector<unsigned char> buf(e * (size_t)K);
                    if (cudaSetDevice(P->device) != cudaSuccess ||
                        cudaMemcpy(buf.data(), (const unsigned char*)d.table + e * (size_t)d.slot_host[arg] * K, buf.size(),
                                   cudaMemcpyDeviceToHost) != cudaSuccess)
                        return -1;
                    double* o = static_cast<double*>(out);
                    for (int64_t k = 0; k < std::min(K, cap / 2); ++k) {
                        double re, im;
                        if (d.prec == kFP32) {
                            const cxf v = reinterpret_cast<const cxf*>(buf.data())[k];
                            re = v.x, im = v.y;
                        } else if (d.prec == kFP64) {
                            const cxd v = reinterpret_cast<const cxd*>(buf.data())[k];
                            re = v.x, im = v.y;
                        } else {
                            const cx<df> v = reinterpret_cast<const cx<df>*>(buf.data())[k];
                            re = (double)v.x.hi + (double)v.x.lo, im = (double)v.y.hi + (double)v.y.lo;
                        }
                        o[2 * k] = re;
                        o[2 * k + 1] = im;
                    }
                }
                return 2 * K;
            }
            const auto& t = hp.lp[level].table[arg];
            if (t.empty()) return -1;
            const int64_t n = (int64_t)t.size();
            if (out) {
                double* o = static_cast<double*>(out);
                for (int64_t k = 0; k < std::min(n, cap / 2); ++k) {
                    o[2 * k] = t[k].real();
                    o[2 * k + 1] = t[k].imag();
                }
            }
            return 2 * n;
        }
        case HFMM_GET_LEAF_BOX: {
            const int64_t n = (int64_t)hp.leaf_level.size();
            if (out) {
                int32_t* o = static_cast<int32_t*>(out);
                for (int64_t i = 0; i < std::min(n, cap / 2); ++i) {
                    o[2 * i] = hp.leaf_level[i];
                    o[2 * i + 1] = hp.leaf_box[i];
                }
            }
            return 2 * n;
        }
        case HFMM_GET_LEAF_SRC:
        case HFMM_GET_LEAF_TGT: {
            const auto& s = (what == HFMM_GET_LEAF_SRC) ? hp.src_start : hp.tgt_start;
            const auto& c = (what == HFMM_GET_LEAF_SRC) ? hp.src_count : hp.tgt_count;
            const int64_t n = (int64_t)s.size();
            if (out) {
                int32_t* o = static_cast<int32_t*>(out);
                for (int64_t i = 0; i < std::min(n, cap / 2); ++i) {
                    o[2 * i] = s[i];
                    o[2 * i + 1] = c[i];
                }
            }
            return 2 * n;
        }
        default:
            return -1;
    }
}

}  // extern "C"
