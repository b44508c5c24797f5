"""Writes the oracle's Fourier-FMM values at sampled targets of full-size workloads.

Run from the repository root: python tests/golden/make_fullsize_golden.py
It calls only the oracle (oracle/fmm.py, oracle/quadrature.py) and the seeded input
generators; the GPU tests compare the library's float64 and mixed applies with these values
element by element.  For each workload: the oracle plans with the same options as the test,
runs S2M, M2M, M2L and L2L over every box (Section 2), and L2T and the near field only in the
leaf boxes of the sampled targets (Eq. FMM_FinalStep at those targets).
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import fmm as ofmm                      # noqa: E402
from oracle import quadrature as oq                 # noqa: E402
from paper_0911_4114_gb300 import workloads as wl  # noqa: E402

# name -> (workload, n points or None, kappa, eps, plan options, charge seed (index, salt), target seed)
CASES = {
    "sphere262k": ("sphere262k", None, 64.0, 1e-6, dict(), (1, 1), (1, 3)),
    # a 262,144-point ellipsoid at the full-size plan's depth: float32 levels 2-4,
    # double-float level 5, float64 level 6 under the mixed policy
    "ellipsoid262k_d6": ("ellipsoid2m", 262144, 200.0, 1e-4, dict(depth=6), (2, 5), (2, 6)),
}
NTARGETS = 1000


def oracle_at_targets(plan, q, idx):
    t = plan.tree
    lf = t.depth
    qs = q.reshape(len(q), -1)[t.src_perm]
    nrhs = qs.shape[1]
    inv = np.empty_like(t.tgt_perm)
    inv[t.tgt_perm] = np.arange(len(t.tgt_perm))
    pos = inv[idx]                                   # sorted positions of the sampled targets
    ends = t.tgt_start + t.tgt_count
    boxes = np.unique(np.searchsorted(ends, pos, side="right"))
    out = ofmm.p2p(plan, qs, boxes=boxes)
    if lf >= 2:
        mlev = {lf: ofmm.s2m(plan, qs)}
        for l in range(lf, 2, -1):
            mlev[l - 1] = ofmm.m2m(plan, mlev[l], l)
        ilev = {l: ofmm.m2l(plan, mlev[l], l) for l in range(2, lf + 1)}
        llev = {2: ilev[2]}
        for l in range(2, lf):
            llev[l + 1] = ofmm.l2l(plan, llev[l], ilev[l + 1], l)
        out = out + ofmm.l2t(plan, llev[lf], nrhs, boxes=boxes)
    return out[pos][:, 0]


def main():
    for name, (wname, n, kappa, eps, opts, qseed, tseed) in CASES.items():
        t0 = time.time()
        s, t = wl.points(wname, n=n)
        q = wl.charges(len(s), 0, wl.rng(*qseed)).astype(np.complex64).astype(np.complex128)
        idx = np.sort(wl.rng(*tseed).choice(len(t), NTARGETS, replace=False))
        plan = ofmm.Plan(s, t, kappa, eps, precision="mixed", **opts)
        phi = oracle_at_targets(plan, q, idx)
        est = max(lp.rounding_estimate(oq.U_FP64) for lp in plan.levels.values())
        ells = np.array([plan.levels[l].ell for l in sorted(plan.levels)])
        np.savez(os.path.join(os.path.dirname(os.path.abspath(__file__)), f"fullsize_{name}.npz"),
                 idx=idx, phi=phi, lf=plan.lf, ell=ells, est=est)
        print(f"{name}: lf {plan.lf}, l {ells.tolist()}, est {est:.2e}, {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
