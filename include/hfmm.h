/*
 * hfmm.h -- C ABI of the GB300 Fourier-basis Helmholtz FMM apply.
 *
 * The library computes the matrix-vector product of Eq. (HelmholtzMatrixVector)
 * of Cecka & Darve, "Fourier Based Fast Multipole Method for the Helmholtz
 * Equation" (arXiv 0911.4114), generalised to targets x_i that differ from the
 * sources y_j:
 *
 *     phi_i = sum_{j : |x_i - y_j| > 0} q_j exp(i kappa |x_i - y_j|) / |x_i - y_j|
 *
 * by the multilevel FMM of Section 2 (S2M, M2M, M2L, L2L, L2T and the near
 * field of Eq. FMM_FinalStep) on the uniform (theta, phi) Fourier quadratures
 * of Section 3, with the band-limited modified transfer function of Algorithm
 * BMTF and the FFT re-quadrature of Section 3.4.
 *
 * Conventions for every entry point:
 *   - Point arrays are host, row-major (n, 3) float64 (x, y, z per point).
 *   - Charge / potential arrays are DEVICE pointers, row-major (n, R) complex
 *     (interleaved re, im) of the given dtype; R is the number of right-hand
 *     sides.  The caller owns them; the library never keeps them.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     An apply only enqueues work on that stream: it allocates nothing and
 *     does not synchronise.  Concurrent applies on one plan are not allowed
 *     (they share the plan's workspace).
 *   - Errors are returned as hfmm_status; nothing is thrown across the ABI.
 *     hfmm_last_error() gives a thread-local message for the last failure.
 */
#ifndef HFMM_H
#define HFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HFMM_MAX_LEVELS 21
#define HFMM_N_STAGES 8

typedef struct hfmm_plan_s* hfmm_plan_t;

typedef enum {
    HFMM_OK = 0,
    HFMM_ERR_ARG = 1,      /* invalid argument (sizes, NaN, kappa <= 0, eps outside (0, 0.1], ...) */
    HFMM_ERR_CUDA = 2,     /* a CUDA call failed (message in hfmm_last_error) */
    HFMM_ERR_NOMEM = 3,    /* host or device allocation failed at plan time */
    HFMM_ERR_UNSTABLE = 4, /* no far-field level at this eps and precision (HFMM_FLAG_REQUIRE_FAR) */
    HFMM_ERR_TIMEOUT = 5,  /* device watchdog: a kernel gave up a bounded wait (reported by hfmm_query) */
    HFMM_ERR_STATE = 6     /* call not valid for this plan (e.g. apply on a host-only plan) */
} hfmm_status;

typedef enum { HFMM_C64 = 0, HFMM_C128 = 1 } hfmm_dtype;

/* Precision policy.  FP64: every stage in float64.  MIXED: per level the first of float32,
 * double-float (float32 pairs, ~48 bits) and float64 that the planner's round-off estimate
 * allows, never coarser than the level above; near field in float32 with exact grid
 * geometry and double-float tile accumulation when eps >= 1e-6 (from 8 right-hand sides
 * as a tensor-core GEMM form with 3xTF32 split products; with sources = targets and one
 * right-hand side each pair of distinct boxes evaluated once), in double-float for
 * 1e-11 <= eps < 1e-6, in float64 below. */
typedef enum { HFMM_PREC_FP64 = 0, HFMM_PREC_MIXED = 1 } hfmm_precision;

/* Level precisions reported by hfmm_query. */
typedef enum { HFMM_LEVEL_FP64 = 0, HFMM_LEVEL_FP32 = 1, HFMM_LEVEL_DF = 2 /* float32 pairs */ } hfmm_level_precision;

typedef struct {
    /* alpha values tried for each level, in order (Section 3.3.3: |r| = alpha sqrt(3) a_l);
     * a 0 ends the list.  Default {0.8, 0.6, 0, 0}; with this default, eps < 1e-7 uses
     * {0.9, 0.8}.  Only levels with kappa * a_l >= 6 are ever active. */
    double alpha_ladder[4];
    /* per-level target eps_l = eps_scale * eps (default 0.25) */
    double eps_scale;
    /* the tree depth never exceeds the smallest depth at which no box holds more
     * than max_leaf sources or max_leaf targets (default 64); with HFMM_FLAG_ADAPTIVE it
     * also decides which boxes split */
    int max_leaf;
    /* > 0: requested depth (replaces the max_leaf rule; active levels may still stop
     * earlier where the stability rule rejects a level).  0 = use max_leaf. */
    int depth;
    /* 1: root cube given by root = {corner x, corner y, corner z, side}; 0: bounding cube */
    int has_root;
    double root[4];
    hfmm_precision precision;
    /* largest number of right-hand sides an apply may use (workspace size), default 1 */
    int max_rhs;
    /* CUDA device ordinal (default 0); -1 builds a host-only plan (queries only, no apply) */
    int device;
    /* bit flags, HFMM_FLAG_* below (default 0) */
    int flags;
    /* device bytes the plan may spend on the plane-wave tables of a float64 leaf level
     * (E[j][p] = exp(i kappa s_p . (x_j - c_b)) for every point and antipodal sample pair,
     * 16 bytes each, evaluated once at plan time; S2M and L2T then read them instead of
     * evaluating float64 sincos): -1 = up to half of the device memory free at plan time
     * (default), 0 = never, > 0 = at most this many bytes.  Levels in float32 or
     * double-float never use tables. */
    int64_t leaf_table_bytes;
    /* buffer boxes between a box and its interaction list (Section 3.3.3): 1 (default, the
     * common case: |r0| >= 2 a_l, neighbour lists of 3^3 boxes, 316 transfer vectors), 2
     * (|r0| >= 3 a_l: a smaller truncation l and more stable levels for the same eps,
     * neighbour lists of 5^3 boxes, 1206 transfer vectors; no kappa a_l >= 6 limit), or 0:
     * the plan-shape tuner chooses the buffer and the leaf level (at most the deepest stable
     * level) that minimise a cost model of one apply (near-field pairs, plane-wave products,
     * interaction-list entries and re-quadrature samples weighed with per-unit times measured
     * on a GB300, for max_rhs right-hand sides); hfmm_query reports the choice and the
     * predicted times.  The tuned plan equals the plan with that buffer and depth = lf.  With
     * HFMM_FLAG_ADAPTIVE the adaptive trees at the uniform model's leaf level and one level
     * deeper are built and costed, and the cheaper is kept. */
    int buffer;
} hfmm_options;

/* hfmm_options.flags: fail with HFMM_ERR_UNSTABLE instead of planning a pure near field
 * (an O(N M) direct sum) when no level can carry a far field -- kappa a_2 < 6, the
 * round-off rule rejects level 2 in every allowed precision and alpha, or the occupancy
 * depth is below 2. */
#define HFMM_FLAG_REQUIRE_FAR 1
/* hfmm_options.flags: compute the T^{s,LL} transfer tables on the host (OpenMP) instead of on
 * the device (the default when a device is given).  Both follow Algorithm BMTF and the
 * per-row anterpolation of Section 3.3.2 in float64 and agree to round-off. */
#define HFMM_FLAG_HOST_TABLES 2
/* hfmm_options.flags: adaptive octree.  A box above the leaf level lf splits only when it
 * lies above level 2, holds more than max_leaf sources or more than max_leaf targets, or is
 * crowded (it holds a point and the other cubes of its level within Chebyshev distance
 * `buffer` hold more than (2 buffer + 1)^3 max_leaf sources or targets), so leaves lie on
 * several levels (Section 2's tree, refined only where the points are dense).  A leaf of
 * level l < lf then sums at most ((2 buffer + 1)^3 + 1 + l ((2 buffer + 1)^3 - 1)) max_leaf
 * sources directly.
 * S2M and L2T run for the leaves of each level at that level's quadrature; M2L stays between
 * boxes of one level (Section 3's diagonal transfer, unchanged); a target leaf B and a source
 * leaf C interact directly when their ancestors at level min(l_B, l_C) are neighbours.  The
 * plane-wave tables of a float64 leaf level are not used. */
#define HFMM_FLAG_ADAPTIVE 4

typedef struct {
    int64_t ns, nt;
    double kappa, eps;
    int occupancy_depth;   /* depth bound from max_leaf (or the requested depth) */
    int lf;                /* deepest active level; < 2 means no far field (near field = direct sum) */
    int64_t p2p_pairs;     /* target-source pairs of the near field */
    /* per level l = 0..HFMM_MAX_LEVELS-1 (valid for 2 <= l <= lf) */
    int level_nbox[HFMM_MAX_LEVELS];   /* nonempty boxes (valid for 0 <= l <= lf) */
    int level_ell[HFMM_MAX_LEVELS];
    int level_ntheta[HFMM_MAX_LEVELS];
    int64_t level_K[HFMM_MAX_LEVELS];  /* stored samples per signature: sum_n N_phi(theta_n) */
    int level_precision[HFMM_MAX_LEVELS];
    double level_alpha[HFMM_MAX_LEVELS];
    double level_round_est[HFMM_MAX_LEVELS];  /* round-off estimate at the level's precision */
    int level_ilist_total[HFMM_MAX_LEVELS];   /* sum of interaction-list lengths */
    /* device milliseconds of the last apply per stage (filled when timing is on):
     * 0 permute-in, 1 near field, 2 S2M, 3 M2M, 4 M2L, 5 L2L, 6 L2T, 7 permute-out */
    double stage_ms[HFMM_N_STAGES];
    int64_t workspace_bytes;
    /* arithmetic of the near field: HFMM_LEVEL_FP32 (float32 exact-grid form, mixed policy
     * with eps >= 1e-6), HFMM_LEVEL_DF (double-float, mixed policy with 1e-11 <= eps < 1e-6)
     * or HFMM_LEVEL_FP64 (float64 policy, or eps < 1e-11) */
    int near_precision;
    /* target-source pairs inside one leaf box (part of p2p_pairs) */
    int64_t p2p_self_pairs;
    /* 1 when sources = targets and the near field evaluates each pair of distinct
     * neighbouring boxes once for both directions (float32 near field, one RHS) */
    int near_symmetric;
    /* 1 when S2M / L2T of the (float64) leaf level read plane-wave tables built at plan time */
    int leaf_tables;
    int64_t leaf_table_bytes;   /* device bytes of those tables (0 without) */
    int buffer;                 /* buffer boxes of the plan (1 or 2) */
    int tuned;                  /* 1 when the plan-shape tuner chose buffer and lf */
    /* the tuner's predicted apply time in ms for [buffer][leaf level] (0: not a candidate) */
    double predicted_ms[3][HFMM_MAX_LEVELS];
    /* symmetric near field: the register budget (resident blocks per SM, 5-8) the plan timed
     * fastest on its own near field at plan time (0: not the symmetric kernel) */
    int near_variant;
    /* tcgen05 near field (float32, 16 or more right-hand sides): (128-target chunk, 16-source
     * tile) pairs of the apply per 64-RHS pass, each 12 MMAs of 128 x 128 x 8 (0: not built) */
    int64_t near_mma_tiles;
    /* 1 for an adaptive tree (HFMM_FLAG_ADAPTIVE); leaves in all and per level (a uniform
     * tree's leaves are the level-lf boxes) */
    int adaptive;
    int64_t nleaf;
    int level_nleaf[HFMM_MAX_LEVELS];
} hfmm_info;

/* Fill *opt with the defaults listed above. */
void hfmm_default_options(hfmm_options* opt);

/* Plan stage (host, float64; Sections 2.1, 3.3, 3.4 and the tree of Section 2).
 * sources: host (ns, 3) float64, ns >= 1.  targets: host (nt, 3) float64, nt >= 1; it
 * may be the same pointer as sources.  kappa > 0; 0 < eps <= 0.1.  opt may be NULL.
 * Builds the octree (level uniform, or adaptive with HFMM_FLAG_ADAPTIVE), the interaction
 * lists and the leaves' near lists, the per-level truncation
 * (Eq. EBF refined by Eq. CollinoError), N_theta (Algorithm Ntheta), N_phi(theta_n)
 * (Algorithm Nphi) and the T^{s,LL} tables of the vectors the lists use (Algorithm BMTF;
 * canonical vectors computed, reflected into the others), copies the points, and (device >= 0) uploads everything and allocates the apply
 * workspace on the device.  On success *out owns all of it; release with hfmm_destroy.
 * Errors: HFMM_ERR_ARG, HFMM_ERR_NOMEM, HFMM_ERR_CUDA, HFMM_ERR_UNSTABLE (only with
 * HFMM_FLAG_REQUIRE_FAR: no level carries a far field). */
hfmm_status hfmm_plan(const double* sources, int64_t ns, const double* targets, int64_t nt,
                      double kappa, double eps, const hfmm_options* opt, hfmm_plan_t* out);

/* Apply (device; Section 2 steps on the Section 3 quadratures).
 * q: device (ns, nrhs) complex of dtype; phi: device (nt, nrhs) complex of dtype,
 * overwritten with the FMM approximation of the sum above.  1 <= nrhs <= max_rhs.
 * Enqueued on `stream` (kernels and, for the symmetric near field, a zero fill of the
 * plan's workspace); no allocation, no synchronisation.
 * Errors: HFMM_ERR_ARG (bad pointer/size/dtype), HFMM_ERR_STATE (host-only plan),
 * HFMM_ERR_CUDA (launch failure). */
hfmm_status hfmm_apply(hfmm_plan_t plan, const void* q, void* phi, int nrhs, hfmm_dtype dtype,
                       void* stream);

/* Adjoint apply: out = A^H w = conj(A^T conj(w)), A the FMM operator of hfmm_apply, by the
 * transposed FMM (each stage of Section 2 transposed: near field with the roles of sources
 * and targets exchanged, transposed L2T, transposed L2L (interpolation in place of
 * anterpolation, Section 3.4 steps reversed), M2L with the opposite transfer vector,
 * transposed M2M, transposed S2M).  It is the exact transpose of the apply's arithmetic,
 * so <A x, y> = <x, A^H y> to round-off.
 * w: device (nt, nrhs) complex of dtype; out: device (ns, nrhs) complex of dtype,
 * overwritten.  Same rules as hfmm_apply (shares its workspace; do not overlap them).
 * Stage times (hfmm_query) are stored in the same slots: near field, transposed L2T,
 * transposed L2L, transposed M2L, transposed M2M, transposed S2M.
 * Errors: HFMM_ERR_ARG, HFMM_ERR_STATE, HFMM_ERR_CUDA. */
hfmm_status hfmm_apply_adjoint(hfmm_plan_t plan, const void* w, void* out, int nrhs, hfmm_dtype dtype,
                               void* stream);

/* Position gradient of the apply (vector-Jacobian product for a real loss L, complex
 * autograd convention g = dL/d conj(phi), e.g. g = 2 (phi - phi*) for L = sum |phi - phi*|^2):
 *   grad[j, c] = Re sum_r q_jr ( sum_k i kappa s_k,c exp(i kappa s_k.(y_j - c_b)) Lambda_b,r(k)
 *                               + sum_{i in N(b)} conj(g_ir) dG(x_i, y_j)/dy_j,c )
 * where Lambda is the transposed far-field chain of hfmm_apply_adjoint applied to conj(g)
 * (s-weighted transposed S2M: the derivative of S2M's plane waves) and dG/dy =
 * G (i kappa - 1/R) (y - x)/R is the near-field kernel derivative.  It is the exact
 * derivative of the FMM approximation with the plan's tree held fixed.
 * q: device (ns, nrhs); g: device (nt, nrhs), complex of dtype; grad: device (ns, 3)
 * float64, overwritten.  Same rules as hfmm_apply.  Errors: HFMM_ERR_ARG, HFMM_ERR_STATE,
 * HFMM_ERR_CUDA. */
hfmm_status hfmm_grad_sources(hfmm_plan_t plan, const void* q, const void* g, double* grad, int nrhs,
                              hfmm_dtype dtype, void* stream);

/* Many independent problems applied by one graph launch (batching of uneven problems).
 * Each problem has its own sources, targets, kappa and eps; all share the options. */
typedef struct hfmm_batch_s* hfmm_batch_t;
typedef struct {
    const double* sources;  /* host (ns, 3) float64 */
    int64_t ns;
    const double* targets;  /* host (nt, 3) float64, may alias sources */
    int64_t nt;
    double kappa;
    double eps;
} hfmm_problem;

/* Plans every problem as hfmm_plan does (the options apply to all of them).  Errors as
 * hfmm_plan; on error nothing is left allocated. */
hfmm_status hfmm_plan_batch(int nprob, const hfmm_problem* problems, const hfmm_options* opt,
                            hfmm_batch_t* out);

/* Applies problem p to q[p] -> phi[p] for every p with ONE cudaGraphLaunch on `stream`.
 * q, phi: host arrays of nprob device pointers ((ns_p, nrhs) and (nt_p, nrhs) complex of
 * dtype).  The graph (every problem's stage kernels, problems spread over concurrent
 * branches) is captured on the first call for a given set of pointers, nrhs and dtype and
 * replayed afterwards; a call with different pointers re-captures.  The first call also
 * runs each problem once outside the graph, on `stream`.  Concurrent calls on one batch
 * are not allowed.  Errors: HFMM_ERR_ARG, HFMM_ERR_STATE, HFMM_ERR_CUDA. */
hfmm_status hfmm_apply_batch(hfmm_batch_t batch, const void* const* q, void* const* phi, int nrhs,
                             hfmm_dtype dtype, void* stream);

/* Number of problems and the plan of problem p (owned by the batch; do not destroy it). */
hfmm_status hfmm_batch_plan(hfmm_batch_t batch, int p, hfmm_plan_t* plan);

/* Releases every plan and the cached graph.  NULL is accepted. */
hfmm_status hfmm_batch_destroy(hfmm_batch_t batch);

/* Plan summary and the per-stage times of the last timed apply.  Synchronises with the
 * device to read the plan's watchdog flag: when a kernel of an earlier call gave up one of
 * its bounded waits (about one second; the tcgen05 near field waits on an mbarrier for its
 * MMAs), the call returns HFMM_ERR_TIMEOUT once and clears the flag -- that call's results
 * are incomplete, the context stays usable.  Errors: HFMM_ERR_ARG, HFMM_ERR_CUDA,
 * HFMM_ERR_TIMEOUT. */
hfmm_status hfmm_query(hfmm_plan_t plan, hfmm_info* info);

/* 1: record per-stage CUDA events in later applies (read with hfmm_query after the
 * stream is synchronised); 0: off (default).  Errors: HFMM_ERR_ARG, HFMM_ERR_STATE. */
hfmm_status hfmm_set_timing(hfmm_plan_t plan, int on);

/* Release the plan and every host/device buffer it owns.  NULL is accepted. */
hfmm_status hfmm_destroy(hfmm_plan_t plan);

/* Thread-local message describing the last failure on this thread ("" if none). */
const char* hfmm_last_error(void);

/* Read-only access to plan internals for tests (host copies).  Returns the number of
 * elements available (copies min(count, cap) of them into out when out != NULL), or -1
 * for an unknown request.  `level` selects the tree level; `arg` is the transfer-vector
 * index for HFMM_GET_TABLE.  Element types: int32 for indices, int64 for permutations,
 * float64 for the interleaved complex table. */
typedef enum {
    HFMM_GET_BOX_IDX = 0,      /* int32 (nbox, 3) box coordinates of `level` */
    HFMM_GET_BOX_PARENT = 1,   /* int32 (nbox) parent position in level-1 */
    HFMM_GET_ILIST_OFF = 2,    /* int32 (nbox+1) CSR offsets of the interaction lists */
    HFMM_GET_ILIST_IDX = 3,    /* int32 interaction-list box positions */
    HFMM_GET_ILIST_V = 4,      /* int32 transfer-vector indices (di+D)*W*W+(dj+D)*W+(dk+D), D = 2b+1,
                                  W = 2D+1 for b buffer boxes (b = 1: (di+3)*49+(dj+3)*7+(dk+3)) */
    HFMM_GET_NLIST_OFF = 5,    /* int32 (nleaf+1) CSR offsets of the leaf near lists (uniform tree:
                                  the neighbours within Chebyshev distance <= b) */
    HFMM_GET_NLIST_IDX = 6,    /* int32 near-list leaf indices */
    HFMM_GET_SRC_PERM = 7,     /* int64 (ns) original index of each sorted source */
    HFMM_GET_TGT_PERM = 8,     /* int64 (nt) original index of each sorted target */
    HFMM_GET_NPHI = 9,         /* int32 (ntheta/2+1) N_phi(theta_n) of `level` */
    HFMM_GET_TABLE = 10,       /* float64 (K, 2) T^{s,LL} of `level` for vector `arg` (device-computed
                                  tables are copied back and converted) */
    HFMM_GET_LEAF_SRC = 11,    /* int32 (nleaf, 2) first sorted source and count per leaf */
    HFMM_GET_LEAF_TGT = 12,    /* int32 (nleaf, 2) first sorted target and count per leaf */
    HFMM_GET_LEAF_BOX = 13     /* int32 (nleaf, 2) level and position in that level of every leaf,
                                  in Morton order (the order of the near lists) */
} hfmm_get;

int64_t hfmm_debug_get(hfmm_plan_t plan, int what, int level, int64_t arg, void* out, int64_t cap);

/* Test support for the device watchdog: enqueues on `stream` one kernel that waits on an
 * mbarrier nothing completes, gives up after the bounded wait (about one second) and sets the
 * plan's watchdog flag, as a tcgen05 kernel whose MMAs never complete would; the next
 * hfmm_query then returns HFMM_ERR_TIMEOUT.  No fault, no hang.  Errors: HFMM_ERR_ARG,
 * HFMM_ERR_STATE (host-only plan), HFMM_ERR_CUDA. */
hfmm_status hfmm_debug_watchdog_probe(hfmm_plan_t plan, void* stream);

/* Test support for allocation failures: after `after` more allocation points of the host
 * planner in the calling thread (the planning stages: bounding cube, occupancy depth, level
 * plans, tree and lists, each level's transfer tables), the next one fails as a host
 * allocation failure would, and hfmm_plan returns HFMM_ERR_NOMEM having released everything
 * it allocated; the hook is then off again.  A countdown that has not fired carries over to
 * the next plan.  after < 0 turns the hook off (the default).  No device call is made.
 * Errors: none (always HFMM_OK). */
hfmm_status hfmm_debug_fail_host_alloc(int after);

/* Largest ns + nt that hfmm_direct_noalloc accepts. */
#define HFMM_NOALLOC_MAX_POINTS (1 << 19)

/* Direct near-field sum for callers that cannot allocate device memory.  The paper has
 * no counterpart: this is a library service.  Some callers cannot call cudaMalloc -- code
 * inside a host framework's operator whose device memory may only come from the
 * framework's own pool (an allocation behind the pool's back escapes its accounting and
 * memory limit), or code on a latency-critical path, where a device allocation is an
 * implicit synchronisation point between streams.  They have no plan (creating one
 * allocates), so this entry point takes everything as device pointers and allocates
 * nothing:
 *   sources (ns, 3), targets (nt, 3): device float64, row-major;
 *   q (ns, nrhs), phi (nt, nrhs): device complex of dtype; phi is overwritten with
 *   sum_{j : R_ij > 0} q_j exp(i kappa R_ij) / R_ij over ALL sources (O(ns * nt) work),
 *   computed with the mixed-precision near-field arithmetic of the planned apply (exact
 *   float32 grid coordinates, float64 accumulation of float32 tile sums).
 * Its only extra device memory is a fixed file-scope __device__ array of 256 bytes plus
 * 32 bytes per point for HFMM_NOALLOC_MAX_POINTS points (16 MiB), which every GPU that
 * loads the library holds until the process exits.  ns + nt above the limit returns
 * HFMM_ERR_ARG with a message.  The first call on a device resolves the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  Every call shares the array, so calls that overlap on the GPU
 * (other streams, other threads) race and must be serialised by the caller.  Enqueued on
 * `stream`; no synchronisation.  A CUDA error already pending when the call starts is
 * reported (HFMM_ERR_CUDA) and left in place; nothing is launched then.
 * Errors: HFMM_ERR_ARG, HFMM_ERR_CUDA. */
hfmm_status hfmm_direct_noalloc(const double* sources, int64_t ns, const double* targets, int64_t nt,
                                const void* q, void* phi, int nrhs, hfmm_dtype dtype, double kappa,
                                void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HFMM_H */
