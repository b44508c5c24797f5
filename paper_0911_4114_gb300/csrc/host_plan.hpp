// Host-side plan of the Fourier-basis FMM: tree, lists, per-level quadratures and
// transfer tables.  Built in float64 on the host by planner.cpp; device.cu uploads it.
#pragma once
#include <array>
#include <complex>
#include <cstdint>
#include <string>
#include <vector>

namespace hfmm {

using cd = std::complex<double>;

constexpr int kMaxLevels = 21;
constexpr int kTreeBits = 20;        // deepest depth the tree code supports
// transfer-vector offsets of b buffer boxes lie in [-D, D]^3, D = 2b + 1; index
// v = (di + D) W^2 + (dj + D) W + (dk + D), W = 2D + 1 (b = 1: 343 slots, 316 vectors;
// b = 2: 1331 slots, 1206 vectors)
inline int transfer_span(int buffer) { return 2 * buffer + 1; }
inline int transfer_width(int buffer) { return 2 * transfer_span(buffer) + 1; }
inline int transfer_slots(int buffer) { int w = transfer_width(buffer); return w * w * w; }

// level arithmetic: float64, float32, or double-float (float32 pairs, mixed policy only)
enum LevelPrec { kFP64 = 0, kFP32 = 1, kDF = 2 };

// Quadrature of one level: rows n = 0..ntheta/2 with nphi[n] points each (Section 3.4's K).
struct Quadrature {
    int ell = 0;
    int ntheta = 0;
    std::vector<int> nphi;         // ntheta/2 + 1 entries, multiples of 4
    std::vector<int64_t> off;      // row offsets, ntheta/2 + 2 entries
    int64_t K = 0;
    void finalize();
};

struct LevelPlan {
    double a = 0, alpha = 0, r = 0, r0 = 0, eps_abs = 0, est = 0;
    int prec = kFP64;
    Quadrature quad;
    // T^{s,LL} for each transfer-vector slot (empty where the level's lists never use it), K each
    std::vector<std::vector<cd>> table;
};

struct TreeLevel {
    std::vector<uint64_t> key;     // Morton keys at this level, ascending
    std::vector<int32_t> idx;      // (n, 3) integer box coordinates
    std::vector<int32_t> parent;   // position of the parent box in the level above
    std::vector<double> center;    // (n, 3)
    std::vector<int32_t> child_start, child_count;  // children in the level below (contiguous)
    std::vector<int32_t> ioff, iidx, iv;            // interaction lists (CSR), level >= 2
    std::vector<char> split;                        // the box has children in the level below
    std::vector<int32_t> leaf_pos;                  // positions of this level's leaf boxes
    // adaptive trees: first sorted point and count of every box's subtree (per box)
    std::vector<int32_t> s_start, s_count, t_start, t_count;
    int64_t nbox() const { return (int64_t)key.size(); }
};

struct HostPlan {
    // inputs (copied)
    std::vector<double> src, tgt;  // (n, 3) original order
    int64_t ns = 0, nt = 0;
    double kappa = 0, eps = 0, eps_l = 0;
    // options
    std::vector<double> alphas;
    double eps_scale = 0.25;
    int max_leaf = 64, depth_req = 0, precision = 0;
    // adaptive tree: a box above the depth splits only when it lies above level 2, holds more
    // than max_leaf sources or targets, or is crowded (the other cubes of its level within
    // Chebyshev distance buffer hold more than (2 buffer + 1)^3 max_leaf sources or targets),
    // so leaves lie on several levels; 0 = level uniform
    int adaptive = 0;
    bool host_tables = true;   // false: T^{s,LL} is computed on the device at upload
    int buffer = 1;      // buffer boxes between a box and its interaction list (Section 3.3.3);
                         // 0 on input: chosen by the plan-shape tuner (1 or 2 on output)
    // inputs of the plan-shape tuner's cost model: right-hand sides, near-field arithmetic,
    // sources = targets, bytes allowed for float64 leaf tables (-1: no explicit limit)
    int model_rhs = 1, model_near = 0;
    bool model_sym = false;
    int64_t model_table_bytes = -1;
    // tuner result: 1 when the buffer / leaf level were chosen by the cost model, and the
    // predicted apply time (ms) of every candidate [buffer][leaf level] (0 = not a candidate)
    int tuned = 0;
    double predicted_ms[3][kMaxLevels] = {};
    int has_root = 0;
    double root[4] = {0, 0, 0, 1};
    // tree
    double corner[3] = {0, 0, 0}, side = 1;
    int occ_depth = 0;   // depth bound (max_leaf rule or requested depth)
    int tree_ready = 0;  // the tuner already built the tree of the chosen shape (adaptive trees)
    int lf = 0;          // deepest active level (tree depth used by the apply)
    std::vector<int64_t> src_perm, tgt_perm;
    std::vector<TreeLevel> levels;                  // 0..lf
    // leaves in Morton order of their points (a uniform tree's leaves are the level-lf boxes):
    // level and position in that level, point ranges, and the leaves each one interacts with
    // directly (CSR; uniform: the neighbours within Chebyshev distance buffer)
    std::vector<int32_t> leaf_level, leaf_box;
    std::vector<int32_t> src_start, src_count, tgt_start, tgt_count;  // per leaf
    std::vector<int32_t> noff, nidx;                // leaf near lists (CSR)
    int64_t p2p_pairs = 0;
    int64_t p2p_self_pairs = 0;   // pairs inside one leaf box (target count x source count)
    // per level l = 2..lf
    std::vector<LevelPlan> lp;                      // indexed by level (0, 1 unused)
};

// Builds everything on the host; returns "" on success or an error message.
std::string build_host_plan(HostPlan& hp);

// T^{s,LL} of one level computed on the device (tables.cu): the canonical vectors the level's
// lists use with their Legendre coefficients (Eq. TransferFn), and for every used transfer
// vector, in ascending index order (the compact slot order of the apply), its canonical
// vector and reflection (bit 0: x -> -x, 1: y -> -y, 2: z -> -z, 3: x <-> y).
struct TableJob {
    int ell = 0, nfull = 0;
    double kappa = 0;
    std::vector<cd> coef;          // (ncanon, ell + 1)
    std::vector<double> rhat;      // (ncanon, 3)
    std::vector<int32_t> slot_canon, slot_flags;
    int ncanon() const { return (int)(rhat.size() / 3); }
};
TableJob make_table_job(const LevelPlan& lp, double kappa, int buffer, const std::vector<char>& used);
// Computes the compact table [slot][K] into a new device allocation in the given storage
// (0 float32, 1 float64, 2 double-float pairs); the caller owns *out.  Returns "" or a message.
std::string device_tables(const TableJob& job, const Quadrature& q, int store, void** out, size_t* bytes);

// --- special functions (special.cpp) ----------------------------------------
void sph_jn_all(int nmax, double x, double* out);     // j_0..j_nmax
void sph_yn_all(int nmax, double x, double* out);     // y_0..y_nmax
void bessel_jn_all(int nmax, double x, double* out);  // J_0..J_nmax (integer order)

// thread-local message returned by hfmm_last_error (api.cu)
void set_last_error(const std::string& msg);

// allocation point of the planner: throws std::bad_alloc when the test hook
// (hfmm_debug_fail_host_alloc) counts down to it in this thread
void alloc_point();

// --- helpers shared by the planner and the device-side setup -----------------
bool is_235(int64_t k);
int64_t round_fft(int64_t n, int64_t mult);
}  // namespace hfmm
