"""ctypes binding of libhfmm.so (argument marshalling only; all work runs in the library).

The library must have been built in-tree (``paper_0911_4114_gb300.build.build()``);
loading fails loudly otherwise -- there is no fallback implementation.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhfmm.so")

MAX_LEVELS = 21
N_STAGES = 8
STAGES = ("permute_in", "near_field", "s2m", "m2m", "m2l", "l2l", "l2t", "permute_out")

OK, ERR_ARG, ERR_CUDA, ERR_NOMEM, ERR_UNSTABLE, ERR_TIMEOUT, ERR_STATE = range(7)
C64, C128 = 0, 1
FLAG_REQUIRE_FAR = 1
FLAG_HOST_TABLES = 2
FLAG_ADAPTIVE = 4
PREC_FP64, PREC_MIXED = 0, 1

GET = dict(BOX_IDX=0, BOX_PARENT=1, ILIST_OFF=2, ILIST_IDX=3, ILIST_V=4, NLIST_OFF=5, NLIST_IDX=6,
           SRC_PERM=7, TGT_PERM=8, NPHI=9, TABLE=10, LEAF_SRC=11, LEAF_TGT=12, LEAF_BOX=13)

EXPORTS = ("hfmm_default_options", "hfmm_plan", "hfmm_apply", "hfmm_query", "hfmm_set_timing",
           "hfmm_destroy", "hfmm_last_error", "hfmm_debug_get", "hfmm_direct_noalloc", "hfmm_apply_adjoint", "hfmm_grad_sources", "hfmm_plan_batch",
           "hfmm_apply_batch", "hfmm_batch_plan", "hfmm_batch_destroy", "hfmm_debug_watchdog_probe",
           "hfmm_debug_fail_host_alloc")
NOALLOC_MAX_POINTS = 1 << 19


class Options(ctypes.Structure):
    _fields_ = [("alpha_ladder", ctypes.c_double * 4), ("eps_scale", ctypes.c_double),
                ("max_leaf", ctypes.c_int), ("depth", ctypes.c_int), ("has_root", ctypes.c_int),
                ("root", ctypes.c_double * 4), ("precision", ctypes.c_int), ("max_rhs", ctypes.c_int),
                ("device", ctypes.c_int), ("flags", ctypes.c_int), ("leaf_table_bytes", ctypes.c_int64),
                ("buffer", ctypes.c_int)]


class Problem(ctypes.Structure):
    _fields_ = [("sources", ctypes.c_void_p), ("ns", ctypes.c_int64), ("targets", ctypes.c_void_p),
                ("nt", ctypes.c_int64), ("kappa", ctypes.c_double), ("eps", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("ns", ctypes.c_int64), ("nt", ctypes.c_int64), ("kappa", ctypes.c_double),
                ("eps", ctypes.c_double), ("occupancy_depth", ctypes.c_int), ("lf", ctypes.c_int),
                ("p2p_pairs", ctypes.c_int64),
                ("level_nbox", ctypes.c_int * MAX_LEVELS), ("level_ell", ctypes.c_int * MAX_LEVELS),
                ("level_ntheta", ctypes.c_int * MAX_LEVELS), ("level_K", ctypes.c_int64 * MAX_LEVELS),
                ("level_precision", ctypes.c_int * MAX_LEVELS), ("level_alpha", ctypes.c_double * MAX_LEVELS),
                ("level_round_est", ctypes.c_double * MAX_LEVELS),
                ("level_ilist_total", ctypes.c_int * MAX_LEVELS),
                ("stage_ms", ctypes.c_double * N_STAGES), ("workspace_bytes", ctypes.c_int64),
                ("near_precision", ctypes.c_int), ("p2p_self_pairs", ctypes.c_int64),
                ("near_symmetric", ctypes.c_int), ("leaf_tables", ctypes.c_int),
                ("leaf_table_bytes", ctypes.c_int64), ("buffer", ctypes.c_int), ("tuned", ctypes.c_int),
                ("predicted_ms", (ctypes.c_double * MAX_LEVELS) * 3), ("near_variant", ctypes.c_int), ("near_mma_tiles", ctypes.c_int64),
                ("adaptive", ctypes.c_int), ("nleaf", ctypes.c_int64), ("level_nleaf", ctypes.c_int * MAX_LEVELS)]


_lib = None


def lib():
    """Load libhfmm.so once; raise if it was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_0911_4114_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
    L.hfmm_default_options.argtypes = [ctypes.POINTER(Options)]
    L.hfmm_default_options.restype = None
    L.hfmm_plan.argtypes = [vp, i64, vp, i64, dbl, dbl, ctypes.POINTER(Options), ctypes.POINTER(vp)]
    L.hfmm_plan.restype = ctypes.c_int
    L.hfmm_apply.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, vp]
    L.hfmm_apply.restype = ctypes.c_int
    L.hfmm_apply_adjoint.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, vp]
    L.hfmm_apply_adjoint.restype = ctypes.c_int
    L.hfmm_grad_sources.argtypes = [vp, vp, vp, vp, ctypes.c_int, ctypes.c_int, vp]
    L.hfmm_grad_sources.restype = ctypes.c_int
    L.hfmm_plan_batch.argtypes = [ctypes.c_int, ctypes.POINTER(Problem), ctypes.POINTER(Options), ctypes.POINTER(vp)]
    L.hfmm_plan_batch.restype = ctypes.c_int
    L.hfmm_apply_batch.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, vp]
    L.hfmm_apply_batch.restype = ctypes.c_int
    L.hfmm_batch_plan.argtypes = [vp, ctypes.c_int, ctypes.POINTER(vp)]
    L.hfmm_batch_plan.restype = ctypes.c_int
    L.hfmm_batch_destroy.argtypes = [vp]
    L.hfmm_batch_destroy.restype = ctypes.c_int
    L.hfmm_query.argtypes = [vp, ctypes.POINTER(Info)]
    L.hfmm_query.restype = ctypes.c_int
    L.hfmm_set_timing.argtypes = [vp, ctypes.c_int]
    L.hfmm_set_timing.restype = ctypes.c_int
    L.hfmm_destroy.argtypes = [vp]
    L.hfmm_destroy.restype = ctypes.c_int
    L.hfmm_last_error.argtypes = []
    L.hfmm_last_error.restype = ctypes.c_char_p
    L.hfmm_debug_get.argtypes = [vp, ctypes.c_int, ctypes.c_int, i64, vp, i64]
    L.hfmm_debug_get.restype = i64
    L.hfmm_direct_noalloc.argtypes = [vp, i64, vp, i64, vp, vp, ctypes.c_int, ctypes.c_int, dbl, vp]
    L.hfmm_direct_noalloc.restype = ctypes.c_int
    L.hfmm_debug_watchdog_probe.argtypes = [vp, vp]
    L.hfmm_debug_watchdog_probe.restype = ctypes.c_int
    L.hfmm_debug_fail_host_alloc.argtypes = [ctypes.c_int]
    L.hfmm_debug_fail_host_alloc.restype = ctypes.c_int
    _lib = L
    return L


class HfmmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"hfmm status {status}: {msg}")
        self.status = status


def check(status):
    if status != OK:
        raise HfmmError(status, lib().hfmm_last_error().decode(errors="replace"))
