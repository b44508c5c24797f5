"""Python face of the C ABI: FmmPlan(sources, targets, kappa, eps, ...).apply(q).

Argument marshalling only.  Device buffers are torch tensors (PyTorch supplies memory and
streams); every step of the apply runs inside libhfmm.so.
"""
import ctypes

import numpy as np

from . import _native as nat
from ._native import MAX_LEVELS


_PREC_NAMES = {0: "fp64", 1: "fp32", 2: "df"}   # hfmm_level_precision codes

def make_options(precision="fp64", alphas=None, eps_scale=0.25, max_leaf=64, depth=0, root=None,
                 max_rhs=1, device=0, require_far=False, leaf_table_bytes=-1, buffer=1, host_tables=False,
                 adaptive=False):
    opt = nat.Options()
    nat.lib().hfmm_default_options(ctypes.byref(opt))
    if alphas is not None:              # None keeps the library default ladder
        for i in range(4):
            opt.alpha_ladder[i] = alphas[i] if i < len(alphas) else 0.0
    opt.eps_scale = eps_scale
    opt.max_leaf = max_leaf
    opt.depth = depth
    if root is not None:
        opt.has_root = 1
        for i in range(4):
            opt.root[i] = float(root[i])
    opt.precision = {"fp64": nat.PREC_FP64, "mixed": nat.PREC_MIXED}[precision]
    opt.max_rhs = max_rhs
    opt.device = device
    opt.flags = ((nat.FLAG_REQUIRE_FAR if require_far else 0) | (nat.FLAG_HOST_TABLES if host_tables else 0)
                 | (nat.FLAG_ADAPTIVE if adaptive else 0))
    opt.leaf_table_bytes = int(leaf_table_bytes)
    opt.buffer = int(buffer)
    return opt


class FmmPlan:
    """Plan of the FMM apply for fixed sources, targets, kappa and eps.

    precision: "fp64" (every stage float64) or "mixed" (per level float32, double-float or
    float64, the first the planner's round-off estimate allows; the near field in float32,
    double-float or float64 by eps).  device=-1 builds a host-only plan (queries only).
    require_far: raise (HFMM_ERR_UNSTABLE) instead of planning a pure near field.
    leaf_table_bytes: device bytes allowed for the plane-wave tables of a float64 leaf level
    (-1: up to half the free device memory, 0: none).
    host_tables: compute the transfer tables on the host (default: on the device when there is one).
    buffer: buffer boxes between a box and its interaction list, 1 or 2 (Section 3.3.3), or 0:
    chosen with the leaf level by the plan's cost model (the "auto" plan shape).
    adaptive: adaptive octree -- boxes split only where they or their neighbourhood hold more
    than max_leaf points per box, so leaves lie on several levels (S2M / L2T per leaf level,
    same-level M2L, direct interaction between leaves whose ancestors at the coarser leaf level
    neighbour).
    """

    def __init__(self, sources, targets, kappa, eps, precision="fp64", alphas=None,
                 eps_scale=0.25, max_leaf=64, depth=0, root=None, max_rhs=1, device=0,
                 require_far=False, leaf_table_bytes=-1, buffer=1, host_tables=False, adaptive=False):
        L = nat.lib()
        src = np.ascontiguousarray(sources, dtype=np.float64).reshape(-1, 3)
        tgt = np.ascontiguousarray(targets, dtype=np.float64).reshape(-1, 3)
        self.same = sources is targets
        opt = make_options(precision, alphas, eps_scale, max_leaf, depth, root, max_rhs, device,
                           require_far, leaf_table_bytes, buffer, host_tables, adaptive)
        h = ctypes.c_void_p()
        nat.check(L.hfmm_plan(src.ctypes.data, src.shape[0], tgt.ctypes.data, tgt.shape[0],
                              float(kappa), float(eps), ctypes.byref(opt), ctypes.byref(h)))
        self._h = h
        self.ns, self.nt = src.shape[0], tgt.shape[0]
        self.max_rhs = max_rhs
        self.precision = precision
        self.device = device

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            nat.lib().hfmm_destroy(h)
            self._h = None

    def close(self):
        self.__del__()

    # -- apply ---------------------------------------------------------------
    def apply_ptr(self, q_ptr, phi_ptr, nrhs, dtype, stream_ptr=0):
        """Raw C-ABI call: device pointers (ints), nrhs, dtype (0 = c64, 1 = c128), stream."""
        nat.check(nat.lib().hfmm_apply(self._h, q_ptr, phi_ptr, int(nrhs), int(dtype), stream_ptr))

    def apply(self, q, out=None, stream=None):
        """phi = A q for a CUDA complex64/complex128 tensor q of shape (ns,) or (ns, R)."""
        import torch
        if not q.is_cuda:
            raise ValueError("q must be a CUDA tensor")
        if q.dtype not in (torch.complex64, torch.complex128):
            raise ValueError("q must be complex64 or complex128")
        single = q.dim() == 1
        q2 = q.reshape(q.shape[0], -1).contiguous()
        if q2.shape[0] != self.ns:
            raise ValueError(f"q has {q2.shape[0]} rows, plan has {self.ns} sources")
        r = q2.shape[1]
        if out is None:
            out = torch.empty((self.nt, r), dtype=q.dtype, device=q.device)
        elif out.shape != (self.nt, r) or out.dtype != q.dtype or not out.is_contiguous():
            raise ValueError("out must be a contiguous (nt, R) tensor of q's dtype")
        st = stream if stream is not None else torch.cuda.current_stream(q.device)
        dtype = nat.C64 if q.dtype == torch.complex64 else nat.C128
        self.apply_ptr(q2.data_ptr(), out.data_ptr(), r, dtype, st.cuda_stream)
        return out[:, 0] if single else out

    def apply_adjoint_ptr(self, w_ptr, out_ptr, nrhs, dtype, stream_ptr=0):
        nat.check(nat.lib().hfmm_apply_adjoint(self._h, w_ptr, out_ptr, int(nrhs), int(dtype), stream_ptr))

    def apply_adjoint(self, w, out=None, stream=None):
        """A^H w for a CUDA complex64/complex128 tensor w of shape (nt,) or (nt, R)."""
        import torch
        if not w.is_cuda or w.dtype not in (torch.complex64, torch.complex128):
            raise ValueError("w must be a CUDA complex64/complex128 tensor")
        single = w.dim() == 1
        w2 = w.reshape(w.shape[0], -1).contiguous()
        if w2.shape[0] != self.nt:
            raise ValueError(f"w has {w2.shape[0]} rows, plan has {self.nt} targets")
        r = w2.shape[1]
        if out is None:
            out = torch.empty((self.ns, r), dtype=w.dtype, device=w.device)
        elif out.shape != (self.ns, r) or out.dtype != w.dtype or not out.is_contiguous():
            raise ValueError("out must be a contiguous (ns, R) tensor of w's dtype")
        st = stream if stream is not None else torch.cuda.current_stream(w.device)
        dtype = nat.C64 if w.dtype == torch.complex64 else nat.C128
        self.apply_adjoint_ptr(w2.data_ptr(), out.data_ptr(), r, dtype, st.cuda_stream)
        return out[:, 0] if single else out

    def grad_sources(self, q, g, out=None, stream=None):
        """Source-position gradient: Re sum_r q_r * (d phi / d y)^T conj(g_r), shape (ns, 3) float64.

        g = dL/d conj(phi) in complex autograd's convention (2 (phi - phi*) for a squared error).
        """
        import torch
        q2 = q.reshape(q.shape[0], -1).contiguous()
        g2 = g.reshape(g.shape[0], -1).to(q.dtype).contiguous()
        if q2.shape != (self.ns, g2.shape[1]) or g2.shape[0] != self.nt:
            raise ValueError("q must be (ns, R) and g (nt, R)")
        if out is None:
            out = torch.empty((self.ns, 3), dtype=torch.float64, device=q.device)
        st = stream if stream is not None else torch.cuda.current_stream(q.device)
        dtype = nat.C64 if q.dtype == torch.complex64 else nat.C128
        nat.check(nat.lib().hfmm_grad_sources(self._h, q2.data_ptr(), g2.data_ptr(), out.data_ptr(),
                                               q2.shape[1], dtype, st.cuda_stream))
        return out

    # -- queries -------------------------------------------------------------
    def set_timing(self, on=True):
        nat.check(nat.lib().hfmm_set_timing(self._h, 1 if on else 0))

    def info(self):
        inf = nat.Info()
        nat.check(nat.lib().hfmm_query(self._h, ctypes.byref(inf)))
        lf = inf.lf
        levels = {}
        for l in range(2, lf + 1):
            levels[l] = dict(nbox=inf.level_nbox[l], ell=inf.level_ell[l], ntheta=inf.level_ntheta[l],
                             K=inf.level_K[l], alpha=inf.level_alpha[l],
                             precision=_PREC_NAMES[inf.level_precision[l]],
                             round_est=inf.level_round_est[l], ilist_total=inf.level_ilist_total[l])
        return dict(ns=inf.ns, nt=inf.nt, kappa=inf.kappa, eps=inf.eps, occupancy_depth=inf.occupancy_depth,
                    lf=lf, p2p_pairs=inf.p2p_pairs, nbox=[inf.level_nbox[l] for l in range(lf + 1)],
                    levels=levels, stage_ms={nat.STAGES[i]: inf.stage_ms[i] for i in range(nat.N_STAGES)},
                    workspace_bytes=inf.workspace_bytes,
                    near_precision=_PREC_NAMES[inf.near_precision],
                    p2p_self_pairs=inf.p2p_self_pairs, near_symmetric=bool(inf.near_symmetric),
                    leaf_tables=bool(inf.leaf_tables), leaf_table_bytes=inf.leaf_table_bytes,
                    buffer=inf.buffer, tuned=bool(inf.tuned),
                    predicted_ms={(b, l): inf.predicted_ms[b][l] for b in (1, 2)
                                  for l in range(MAX_LEVELS) if inf.predicted_ms[b][l] > 0},
                    near_variant=inf.near_variant, near_mma_tiles=inf.near_mma_tiles,
                    adaptive=bool(inf.adaptive), nleaf=inf.nleaf,
                    level_nleaf=[inf.level_nleaf[l] for l in range(lf + 1)])

    def debug_get(self, what, level=0, arg=0):
        L = nat.lib()
        code = nat.GET[what]
        n = L.hfmm_debug_get(self._h, code, level, arg, None, 0)
        if n < 0:
            raise KeyError((what, level, arg))
        dt = {"SRC_PERM": np.int64, "TGT_PERM": np.int64, "TABLE": np.float64}.get(what, np.int32)
        out = np.zeros(n, dtype=dt)
        L.hfmm_debug_get(self._h, code, level, arg, out.ctypes.data, n)
        if what == "TABLE":
            return out[0::2] + 1j * out[1::2]
        if what == "BOX_IDX":
            return out.reshape(-1, 3)
        if what in ("LEAF_SRC", "LEAF_TGT", "LEAF_BOX"):
            return out.reshape(-1, 2)
        return out


def direct_noalloc(sources, targets, q, kappa, out=None, stream=None):
    """Direct near-field sum through hfmm_direct_noalloc (no device allocation inside).

    sources (ns, 3), targets (nt, 3): CUDA float64 tensors; q: CUDA complex64/128 (ns,) or
    (ns, R), all on one device.  Callers that may not allocate pass `out`, a contiguous
    (nt, R) tensor of q's dtype on that device; without it this wrapper allocates `out`.
    Every shape, dtype and device is checked here, before the native call.
    """
    import torch
    for name, t in (("sources", sources), ("targets", targets)):
        if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or t.dim() != 2 or t.shape[1] != 3:
            raise ValueError(f"{name} must be a contiguous CUDA float64 (n, 3) tensor")
    if not q.is_cuda or q.dtype not in (torch.complex64, torch.complex128):
        raise ValueError("q must be a CUDA complex64/complex128 tensor")
    if q.dim() not in (1, 2):
        raise ValueError("q must have shape (ns,) or (ns, R)")
    if sources.device != q.device or targets.device != q.device:
        raise ValueError("sources, targets and q must be on one device")
    single = q.dim() == 1
    q2 = q.reshape(q.shape[0], -1).contiguous()
    if q2.shape[0] != sources.shape[0]:
        raise ValueError(f"q has {q2.shape[0]} rows, there are {sources.shape[0]} sources")
    r = q2.shape[1]
    nt = targets.shape[0]
    if out is None:
        out = torch.empty((nt, r), dtype=q.dtype, device=q.device)
    elif (out.device != q.device or out.dtype != q.dtype or tuple(out.shape) != (nt, r)
          or not out.is_contiguous()):
        raise ValueError("out must be a contiguous (nt, R) tensor of q's dtype on q's device")
    st = stream if stream is not None else torch.cuda.current_stream(q.device)
    dtype = nat.C64 if q.dtype == torch.complex64 else nat.C128
    nat.check(nat.lib().hfmm_direct_noalloc(sources.data_ptr(), sources.shape[0], targets.data_ptr(),
                                             nt, q2.data_ptr(), out.data_ptr(), r, dtype,
                                             float(kappa), st.cuda_stream))
    return out[:, 0] if single else out


class _BorrowedPlan(FmmPlan):
    """A plan owned by a batch (not destroyed by Python)."""

    def __init__(self, handle, ns, nt, max_rhs):
        self._borrowed = handle
        self.ns, self.nt, self.max_rhs = ns, nt, max_rhs

    def __del__(self):
        pass

    @property
    def _h(self):
        return self._borrowed


class FmmBatch:
    """Independent problems applied by one CUDA graph launch (hfmm_plan_batch / hfmm_apply_batch).

    problems: list of (sources, targets, kappa, eps); options as for FmmPlan.
    """

    def __init__(self, problems, **opts):
        L = nat.lib()
        self._keep = []
        arr = (nat.Problem * len(problems))()
        self.sizes = []
        for i, (s, t, kappa, eps) in enumerate(problems):
            s = np.ascontiguousarray(s, dtype=np.float64).reshape(-1, 3)
            t = np.ascontiguousarray(t, dtype=np.float64).reshape(-1, 3)
            self._keep += [s, t]
            arr[i] = nat.Problem(s.ctypes.data, s.shape[0], t.ctypes.data, t.shape[0], float(kappa), float(eps))
            self.sizes.append((s.shape[0], t.shape[0]))
        opt = make_options(**opts)
        self.max_rhs = opt.max_rhs
        h = ctypes.c_void_p()
        nat.check(L.hfmm_plan_batch(len(problems), arr, ctypes.byref(opt), ctypes.byref(h)))
        self._h = h
        self._keep = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            nat.lib().hfmm_batch_destroy(h)
            self._h = None

    def plan(self, p):
        ph = ctypes.c_void_p()
        nat.check(nat.lib().hfmm_batch_plan(self._h, p, ctypes.byref(ph)))
        ns, nt = self.sizes[p]
        return _BorrowedPlan(ph, ns, nt, self.max_rhs)

    def apply(self, qs, outs=None, stream=None):
        """qs: list of CUDA (ns_p, R) complex tensors; returns the list of (nt_p, R) results."""
        import torch
        n = len(self.sizes)
        if len(qs) != n:
            raise ValueError(f"need {n} charge tensors")
        q2 = [q.reshape(q.shape[0], -1).contiguous() for q in qs]
        r = q2[0].shape[1]
        dt = q2[0].dtype
        if outs is None:
            outs = [torch.empty((self.sizes[p][1], r), dtype=dt, device=q2[p].device) for p in range(n)]
        qp = (ctypes.c_void_p * n)(*[q.data_ptr() for q in q2])
        op = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
        st = stream if stream is not None else torch.cuda.current_stream(q2[0].device)
        dtype = nat.C64 if dt == torch.complex64 else nat.C128
        nat.check(nat.lib().hfmm_apply_batch(self._h, qp, op, r, dtype, st.cuda_stream))
        return outs
