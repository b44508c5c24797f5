"""Helpers for the GPU tests: run the library's apply on torch CUDA tensors."""
import numpy as np


def run_apply(plan, q, dtype="c128"):
    import torch
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    qt = torch.as_tensor(np.ascontiguousarray(q)).to(device="cuda", dtype=tdt)
    out = plan.apply(qt)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.complex128)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def fp64_parity_tol(oracle_plan):
    """Parity bound between two float64 evaluations of the same plan: both sides round
    an ill-conditioned quadrature sum and compute their transfer tables independently;
    measured element differences run up to ~50x the planner's round-off estimate (largest
    level), so the bound is 256x that estimate, floor 1e-12."""
    from oracle import quadrature as oq
    est = max([lp.rounding_estimate(oq.U_FP64) for lp in oracle_plan.levels.values()] or [0.0])
    return max(1e-12, 256.0 * est)
