"""Helpers for the GPU tests: run the library's apply on torch CUDA tensors."""
import numpy as np

# Element-wise parity bound between the float64 GPU apply and the float64 oracle FMM, in
# units of the planner's float64 round-off estimate of the worst active level (reading of
# the "1e-12 relative" parity target where a level is ill-conditioned); floor 1e-12.
# Measured ratios on a GB300 (max|diff| / (est max|phi|)): 31.7 (4k cube, kappa 8 pi),
# 76.6 (3k cube, kappa 60), 54.9 (two spheres), 2.0 (6k sphere); 128 is the next power of
# two above the largest.
FP64_PARITY_MULT = 128.0


def run_apply(plan, q, dtype="c128"):
    import torch
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    qt = torch.as_tensor(np.ascontiguousarray(q)).to(device="cuda", dtype=tdt)
    out = plan.apply(qt)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.complex128)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def fp64_round_est(oracle_plan):
    """The planner's float64 round-off estimate of the worst active level (0 without levels)."""
    from oracle import quadrature as oq
    return max([lp.rounding_estimate(oq.U_FP64) for lp in oracle_plan.levels.values()] or [0.0])


def fp64_parity_tol(oracle_plan, mult=FP64_PARITY_MULT):
    """Parity bound between two float64 evaluations of the same plan: both sides round the
    same (possibly ill-conditioned) quadrature sums and compute their transfer tables
    independently, so they agree to the round-off of those sums, which the planner's
    estimate measures; the bound is `mult` times that estimate, floor 1e-12."""
    return max(1e-12, mult * fp64_round_est(oracle_plan))


def check_fp64_parity(got, want, oracle_plan, label, mult=FP64_PARITY_MULT):
    """Assert max|got - want| <= tol * max|want| and print the measured ratio to the estimate."""
    est = fp64_round_est(oracle_plan)
    diff = float(np.max(np.abs(got - want)) / np.max(np.abs(want)))
    ratio = diff / est if est > 0 else float("inf")
    tol = fp64_parity_tol(oracle_plan, mult)
    print(f"fp64-parity {label}: max|diff|/max|want| = {diff:.3e}  est = {est:.3e}  "
          f"ratio = {ratio:.2f}  tol = {tol:.3e}")
    assert diff <= tol, (label, diff, est, ratio)
    return diff, est
