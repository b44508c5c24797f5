"""CPU FP64 Fourier-basis FMM, step by step (oracle; test infrastructure only).

Section 2 of the paper (initialisation/S2M, upward pass/M2M, transfer/M2L,
downward pass/L2L, field computation Eq. FMM_FinalStep) carried out on the
Fourier quadratures of Section 3 with the re-quadrature of Section 3.4:

* S2M   M_b(s_k) = sum_{j in b} q_j exp(i k s_k.(y_j - c_b))             (leaf level)
* M2M   M_a += requad_{K_l -> K_{l-1}}(M_b) * exp(i k s.(c_b - c_a))      (interpolate, then shift)
* M2L   I_a = sum_{b in I(a)} T^{s,LL}_{c_b - c_a} * M_b                  (diagonal, per level)
* L2L   L_c = requad_{K_l -> K_{l+1}}(L_a * exp(i k s.(c_a - c_c))) + I_c  (shift, then anterpolate)
* L2T   phi_i = sum_k w_k L_b(s_k) exp(i k s_k.(c_b - x_i))
        w_k = m_n 4 pi^2 / (N_theta N_phi(theta_n)), m_n = 1 on the poles, 2 elsewhere
        (the rows n > N_theta/2 fold onto N_theta - n by Eq. NumSphereSym)
* P2P   phi_i += sum_{j in N(b), R_ij > 0} q_j exp(i k R_ij) / R_ij

On an adaptive tree (tree.py) the leaves lie on several levels: S2M runs for the
leaves of each level at that level's quadrature and is added to the M2M result
(which is zero for a leaf), L2T runs for the leaves of each level, and P2P takes
each leaf's list of directly interacting leaves.

Levels 2..L_f are active (L_f = deepest level the stability rule accepts, never
deeper than the occupancy depth, and only levels whose boxes are about a wavelength
or larger, k a_l >= 6: below that the Gegenbauer series converges only
geometrically for pairs near opposite box corners); when no level is accepted (L_f < 2) the whole
apply is the near field over the level-L_f neighbour lists, i.e. the direct sum.

The stability rule (a reading; the paper only names the low-frequency breakdown
and notes that a lower alpha gives a smaller quadrature):  for each level, top
down, the first alpha of the ladder ((0.8, 0.6), or (0.9, 0.8) for eps < 1e-7)
whose plan passes
    est(u) = u * k|r0| * sqrt(sum_{n<=l} (2n+1)|h_n(k|r0|)|^2) / sqrt(K) <= f_p * eps_l
in one of the precisions the policy allows is taken (u = 2^-53, f = 1/16 for
fp64; u = 2^-48, f = 1/16 for double-float (float32 pairs); u = 2^-24, f = 1 for
fp32; the policy 'fp64' allows fp64 only, 'mixed' tries fp32, then double-float, then
fp64 for a given alpha, and a level never takes a lower precision than the level
above it); the first level that no alpha passes ends the active levels.  est is the relative random round-off of the quadrature sum with
the sphere rms of T (orthogonality of the P_n); f_fp64 = 1/16 because in the
evanescent regime (l > k|r0|, the only place fp64 is ever limited) measured
errors run 17-25x above est, while f_fp32 = 1 because in the propagating regime
(the only place fp32 ever passes) measured table-rounding errors run below est.
"""
import math

import numpy as np

from . import quadrature as qd
from .direct import kernel_matrix
from .tree import Tree, root_cube, occupancy_depth, transfer_offset

PRECISION_UNIT = {'fp64': qd.U_FP64, 'df': qd.U_DF, 'fp32': qd.U_FP32}
# acceptance factor of the stability rule per precision (see module docstring)
PRECISION_FACTOR = {'fp64': 1.0 / 16.0, 'df': 1.0 / 16.0, 'fp32': 1.0}
MIN_KA = 6.0          # one buffer box
MIN_KA_TWO_BUFFER = 0.0


def min_ka(buffer):
    """Smallest k a_l of an active level: 6 with one buffer box (boxes of about a wavelength:
    the Gegenbauer series converges only geometrically, ratio up to alpha sqrt(3)/2, for pairs
    near opposite corners of small boxes); none with two (ratio at most alpha sqrt(3)/3; the
    round-off rule alone decides)."""
    return MIN_KA if buffer == 1 else MIN_KA_TWO_BUFFER


def alpha_ladder(eps):
    """Default alpha ladder: (0.8, 0.6), or (0.9, 0.8) when eps < 1e-7."""
    return (0.9, 0.8) if eps < 1e-7 else (0.8, 0.6)


def level_precisions(policy):
    """Precisions a level may use under a plan policy, in order of preference."""
    return {'fp64': ('fp64',), 'mixed': ('fp32', 'df', 'fp64')}[policy]


class Plan:
    """Everything the apply needs: tree to depth L_f, per-level quadrature, transfer tables."""

    def __init__(self, sources, targets, kappa, eps, alphas=None, max_leaf=64, depth=0,
                 root=None, precision='fp64', eps_scale=0.25, buffer=1, adaptive=False):
        self.sources = np.ascontiguousarray(sources, dtype=np.float64).reshape(-1, 3)
        self.targets = np.ascontiguousarray(targets, dtype=np.float64).reshape(-1, 3)
        self.kappa = float(kappa)
        self.eps = float(eps)
        self.eps_l = eps_scale * self.eps
        self.buffer = int(buffer)
        allp = np.concatenate([self.sources, self.targets], axis=0)
        corner, side = root_cube(allp, root)
        if depth > 0:
            dmax = int(depth)
        else:
            dmax = occupancy_depth(self.sources, self.targets, corner, side, max_leaf)
        self.levels = {}
        self.level_precision = {}
        lf = 1
        allowed = list(level_precisions(precision))
        if alphas is None:
            alphas = alpha_ladder(self.eps)
        for l in range(2, dmax + 1):
            if self.kappa * side / float(2 ** l) < min_ka(self.buffer):
                break
            chosen = None
            for alpha in alphas:
                lp = qd.LevelPlan(self.kappa, side / float(2 ** l), self.eps_l, alpha, self.buffer)
                for p in allowed:
                    if lp.rounding_estimate(PRECISION_UNIT[p]) <= self.eps_l * PRECISION_FACTOR[p]:
                        chosen = (lp, p)
                        break
                if chosen:
                    break
            if chosen is None:
                break
            self.levels[l], self.level_precision[l] = chosen
            # precision never decreases with depth: a deeper level keeps at least this one's
            allowed = allowed[allowed.index(chosen[1]):]
            lf = l
        if dmax < 2:
            lf = dmax
        self.occupancy_depth = dmax
        self.lf = lf
        self.adaptive = bool(adaptive)
        self.tree = Tree(self.sources, self.targets, lf, root, self.buffer,
                         max_leaf if self.adaptive else None)
        self._tables = {}

    def table(self, l, v):
        """T^{s,LL} of level l for transfer-vector index v (computed directly, no symmetry)."""
        key = (l, int(v))
        if key not in self._tables:
            d = transfer_offset(v, self.buffer).astype(np.float64)
            a = self.tree.levels[l]['a']
            lp = self.levels[l]
            self._tables[key] = qd.tsll(lp.ell, self.kappa, d * a, lp.ntheta, lp.nphi)
        return self._tables[key]


def _boxes(boxes, n):
    """All n boxes, or the given subset (used to time the oracle on a sample of boxes)."""
    return range(n) if boxes is None else [int(b) for b in boxes]


def _leaves(lev, boxes):
    """The leaf boxes of a level, or the given subset of its boxes."""
    return np.nonzero(lev['leaf'])[0] if boxes is None else [int(b) for b in boxes]


def s2m(plan, qs, boxes=None, l=None):
    """Signatures M[b, r, k] of the leaves of level l (default: the depth; boxes: optional
    subset; the other boxes stay zero)."""
    t = plan.tree
    lf = t.depth if l is None else l
    quad = plan.levels[lf].quad
    lev = t.levels[lf]
    ys = plan.sources[t.src_perm]
    out = np.zeros((len(lev['key']), qs.shape[1], quad.K), dtype=np.complex128)
    for b in _leaves(lev, boxes):
        s0, sc = lev['src_start'][b], lev['src_count'][b]
        if sc == 0:
            continue
        d = ys[s0:s0 + sc] - lev['center'][b]
        e = np.exp(1j * plan.kappa * (quad.shat @ d.T))    # [K, n]
        out[b] = (e @ qs[s0:s0 + sc]).T
    return out


def m2m(plan, mchild, l, boxes=None):
    """Level l signatures -> level l-1 signatures (boxes: optional subset of children)."""
    t = plan.tree
    qa, qb = plan.levels[l].quad, plan.levels[l - 1].quad
    child, par = t.levels[l], t.levels[l - 1]
    kids = list(_boxes(boxes, len(child['key'])))
    up = qd.requadrature(mchild[kids], qa, qb)             # [nb, R, K_{l-1}]
    out = np.zeros((len(par['key']),) + up.shape[1:], dtype=np.complex128)
    for i, b in enumerate(kids):
        p = child['parent'][b]
        d = child['center'][b] - par['center'][p]
        out[p] += up[i] * np.exp(1j * plan.kappa * (qb.shat @ d))
    return out


def m2l(plan, mlev, l, boxes=None):
    t = plan.tree
    out = np.zeros_like(mlev)
    for a in _boxes(boxes, len(t.levels[l]['key'])):
        for b, v in zip(t.ilist[l][a], t.vlist[l][a]):
            out[a] += plan.table(l, v) * mlev[b]
    return out


def l2l(plan, lpar, ichild, l, boxes=None):
    """Level l locals -> level l+1 locals (plus that level's incoming I); boxes: optional
    subset of children (the result then holds those children only, in that order)."""
    t = plan.tree
    qa, qb = plan.levels[l].quad, plan.levels[l + 1].quad
    child, par = t.levels[l + 1], t.levels[l]
    kids = list(_boxes(boxes, len(child['key'])))
    shifted = np.zeros((len(kids),) + lpar.shape[1:], dtype=np.complex128)
    for i, c in enumerate(kids):
        p = child['parent'][c]
        d = par['center'][p] - child['center'][c]
        shifted[i] = lpar[p] * np.exp(1j * plan.kappa * (qa.shat @ d))
    return qd.requadrature(shifted, qa, qb) + ichild[kids]


def l2t(plan, lleaf, nrhs, boxes=None, l=None):
    """Far field at the targets of the leaves of level l (default: the depth); the other
    targets stay zero."""
    t = plan.tree
    lf = t.depth if l is None else l
    quad = plan.levels[lf].quad
    lev = t.levels[lf]
    xs = plan.targets[t.tgt_perm]
    out = np.zeros((xs.shape[0], nrhs), dtype=np.complex128)
    for b in _leaves(lev, boxes):
        t0, tc = lev['tgt_start'][b], lev['tgt_count'][b]
        if tc == 0:
            continue
        d = lev['center'][b] - xs[t0:t0 + tc]
        e = np.exp(1j * plan.kappa * (d @ quad.shat.T)) * quad.w   # [n, K]
        out[t0:t0 + tc] = e @ lleaf[b].T
    return out


def p2p(plan, qs, boxes=None):
    t = plan.tree
    lf = t.depth
    ys = plan.sources[t.src_perm]
    xs = plan.targets[t.tgt_perm]
    out = np.zeros((xs.shape[0], qs.shape[1]), dtype=np.complex128)
    for b in _boxes(boxes, len(t.leaf_level)):
        t0, tc = t.tgt_start[b], t.tgt_count[b]
        if tc == 0:
            continue
        idx = np.concatenate([np.arange(t.src_start[n], t.src_start[n] + t.src_count[n])
                              for n in t.nlist[b]]).astype(np.int64)
        if idx.size == 0:
            continue
        g = kernel_matrix(xs[t0:t0 + tc], ys[idx], plan.kappa)
        out[t0:t0 + tc] = g @ qs[idx]
    return out


def apply(plan, q, return_stages=False):
    """phi = A q for q of shape (ns,) or (ns, R); the FMM approximation of the direct sum."""
    q = np.asarray(q, dtype=np.complex128)
    single = q.ndim == 1
    q2 = q.reshape(q.shape[0], -1)
    t = plan.tree
    qs = q2[t.src_perm]
    nrhs = q2.shape[1]
    stages = {}
    phi_s = p2p(plan, qs)
    lf = t.depth
    if lf >= 2:
        mlev = {lf: s2m(plan, qs)}
        for l in range(lf, 2, -1):
            mlev[l - 1] = m2m(plan, mlev[l], l)
            if t.levels[l - 1]['leaf'].any():       # leaves above the depth (adaptive tree)
                mlev[l - 1] = mlev[l - 1] + s2m(plan, qs, l=l - 1)
        ilev = {l: m2l(plan, mlev[l], l) for l in range(2, lf + 1)}
        llev = {2: ilev[2]}
        for l in range(2, lf):
            llev[l + 1] = l2l(plan, llev[l], ilev[l + 1], l)
        far = l2t(plan, llev[lf], nrhs)
        for l in range(2, lf):
            if t.levels[l]['leaf'].any():
                far = far + l2t(plan, llev[l], nrhs, l=l)
        stages.update(M=mlev, I=ilev, L=llev, far=far, near=phi_s.copy())
        phi_s = phi_s + far
    phi = np.zeros_like(phi_s)
    phi[t.tgt_perm] = phi_s
    if single:
        phi = phi[:, 0]
    if return_stages:
        return phi, stages
    return phi
