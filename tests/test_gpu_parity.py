"""GPU parity: the CUDA apply (through the C ABI) against the CPU oracle.

FP64 path: element-wise against the oracle FMM on the same plan integers (bound from the
arithmetic, floor 1e-12) and within eps of the direct sum.  Mixed path: within eps of
the direct sum.  Full-size sphere: 1,000 sampled targets against the direct sum.
"""
import zlib

import numpy as np
import pytest

from oracle import direct, fmm as ofmm
from paper_0911_4114_gb300 import FmmPlan, workloads as wl
from gpu_util import check_fp64_parity, fp64_parity_tol, rel, run_apply

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _case(name):
    g = wl.rng(90 + zlib.crc32(name.encode()) % 97)
    if name == "cube4k":                       # the 4,096-point uniform-cube workload
        x, _ = wl.points("cube4k_fp64")
        return x, x, 8 * np.pi, 1e-6, dict(depth=3, root=(0, 0, 0, 1.0))
    if name == "cube_hf":                      # two active levels, high frequency
        x = wl.cube(3000, g)
        return x, x, 60.0, 1e-6, dict(depth=3, root=(0, 0, 0, 1.0))
    if name == "sphere_small":
        x = wl.sphere(6000, g)
        return x, x, 24.0, 1e-6, dict(max_leaf=32)
    if name == "two_spheres":
        s = wl.sphere(2000, g)
        t = wl.sphere(1500, g, radius=1.5)
        return s, t, 12.0, 1e-6, dict(max_leaf=16)
    raise KeyError(name)


@pytest.mark.parametrize("name", ["cube4k", "cube_hf", "sphere_small", "two_spheres"])
def test_fp64_matches_oracle_fmm_and_direct(name):
    s, t, kappa, eps, kw = _case(name)
    q = wl.charges(len(s), 0, wl.rng(7))
    lib = FmmPlan(s, t, kappa, eps, precision="fp64", **kw)
    orc = ofmm.Plan(s, t, kappa, eps, precision="fp64", **kw)
    assert lib.info()["lf"] == orc.lf
    got = run_apply(lib, q)
    want = ofmm.apply(orc, q)
    check_fp64_parity(got, want, orc, name)
    assert rel(got, direct.direct(s, t, q, kappa)) <= eps


def test_fp64_well_conditioned_cube_matches_oracle_to_1e12():
    """The 4,096-point uniform-cube workload on one propagating level (depth 2, root [0,1]^3,
    kappa = 120 so kappa a_2 = 30: the quadrature sum has little cancellation and the
    round-off estimate is ~4e-16).  Here the float64 GPU apply must match the oracle FMM
    element-wise to 1e-12 relative to max|phi| with no round-off allowance."""
    x, _ = wl.points("cube4k_fp64")
    kappa, eps, kw = 120.0, 1e-6, dict(depth=2, root=(0, 0, 0, 1.0))
    q = wl.charges(len(x), 0, wl.rng(7))
    lib = FmmPlan(x, x, kappa, eps, precision="fp64", **kw)
    orc = ofmm.Plan(x, x, kappa, eps, precision="fp64", **kw)
    assert lib.info()["lf"] == orc.lf == 2
    got = run_apply(lib, q)
    want = ofmm.apply(orc, q)
    diff, est = check_fp64_parity(got, want, orc, "cube4k_kappa120_depth2", mult=0.0)
    assert est < 1e-15 and diff <= 1e-12
    assert rel(got, direct.direct(x, x, q, kappa)) <= eps


@pytest.mark.parametrize("name", ["cube4k", "cube_hf", "sphere_small", "two_spheres"])
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_mixed_within_eps_of_direct(name, dtype):
    s, t, kappa, eps, kw = _case(name)
    q = wl.charges(len(s), 0, wl.rng(8))
    lib = FmmPlan(s, t, kappa, eps, precision="mixed", **kw)
    got = run_apply(lib, q, dtype)
    assert rel(got, direct.direct(s, t, q, kappa)) <= eps


def test_multi_rhs_columns_agree():
    s, t, kappa, eps, kw = _case("cube_hf")
    q = wl.charges(len(s), 3, wl.rng(9))
    lib = FmmPlan(s, t, kappa, eps, precision="fp64", max_rhs=4, **kw)
    orc = ofmm.Plan(s, t, kappa, eps, precision="fp64", **kw)
    got = run_apply(lib, q)
    tol = fp64_parity_tol(orc)
    for r in range(3):
        one = run_apply(lib, q[:, r])
        assert np.max(np.abs(one - got[:, r])) <= tol * np.max(np.abs(got))
    assert rel(got, direct.direct(s, t, q, kappa)) <= eps


@pytest.mark.parametrize("n", [1, 2, 7, 65, 300])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ragged_and_tiny_inputs(n, precision):
    g = wl.rng(11, salt=n)
    x = wl.cube(n, g)
    x[n // 2] = x[0]                      # a coincident pair where n > 1
    q = wl.charges(n, 0, g)
    lib = FmmPlan(x, x, 5.0, 1e-6, precision=precision, max_leaf=8)
    got = run_apply(lib, q)
    want = direct.direct(x, x, q, 5.0)
    if not np.any(want):                  # one point, or only a coincident pair: nothing to sum
        assert np.all(got == 0)
    else:
        assert rel(got, want) <= (1e-13 if precision == "fp64" else 1e-6)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sphere262k_sampled_targets(precision):
    """The 262,144-point sphere workload at kappa = 64, eps = 1e-6: 1,000 sampled targets."""
    s, t = wl.points("sphere262k")
    q = wl.charges(len(s), 0, wl.rng(1, salt=1)).astype(np.complex64)
    lib = FmmPlan(s, t, 64.0, 1e-6, precision=precision)
    got = run_apply(lib, q, "c64")
    idx = np.sort(wl.rng(1, salt=2).choice(len(t), 1000, replace=False))
    want = direct.direct(s, t[idx], q.astype(np.complex128), 64.0)
    assert rel(got[idx], want) <= 1e-6


@pytest.mark.parametrize("nrhs", [1, 5])
def test_double_float_near_field_against_direct(nrhs):
    """Mixed policy below eps = 1e-6: the near field runs in double-float.  With one box
    (no far field) the apply is the near field alone, so it must match the float64 direct
    sum to double-float round-off; the transposed near field must match the direct
    adjoint the same way.  R = 5 covers the four-RHS pass and a ragged remainder."""
    g = wl.rng(12, salt=nrhs)
    x = wl.cube(2500, g)
    x[100] = x[7]                                   # a coincident pair: skipped (R = 0)
    q = wl.charges(len(x), nrhs if nrhs > 1 else 0, g)
    lib = FmmPlan(x, x, 30.0, 1e-9, precision="mixed", max_leaf=4096, max_rhs=nrhs)
    info = lib.info()
    assert info["near_precision"] == "df" and info["lf"] < 2
    got = run_apply(lib, q)
    want = direct.direct(x, x, q, 30.0)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
    import torch
    w = wl.charges(len(x), nrhs if nrhs > 1 else 0, g)
    adj = lib.apply_adjoint(torch.as_tensor(w, device="cuda")).cpu().numpy()
    want_adj = direct.direct_adjoint(x, x, w, 30.0)
    assert np.max(np.abs(adj - want_adj)) <= 1e-12 * np.max(np.abs(want_adj))


@pytest.mark.parametrize("name", ["cube_hf", "sphere_small", "two_spheres"])
def test_mixed_tight_eps_within_eps_of_direct(name):
    """eps = 1e-9 under the mixed policy: double-float near field and levels."""
    s, t, kappa, _, kw = _case(name)
    q = wl.charges(len(s), 0, wl.rng(13))
    lib = FmmPlan(s, t, kappa, 1e-9, precision="mixed", **kw)
    assert lib.info()["near_precision"] == "df"
    got = run_apply(lib, q)
    assert rel(got, direct.direct(s, t, q, kappa)) <= 1e-9


@pytest.mark.parametrize("name", ["cube_hf", "sphere_small"])
def test_symmetric_near_field_matches_one_way(name):
    """Sources = targets with one RHS takes the symmetric float32 near field (each pair of
    distinct neighbouring boxes evaluated once, both directions); two RHS take the one-way
    kernel.  Column 0 of the two must agree to float32 round-off (a dropped or doubled
    pair would show at the 1e-2 level), apply and adjoint."""
    import torch
    s, _, kappa, eps, kw = _case(name)
    g = wl.rng(14)
    q = wl.charges(len(s), 2, g)
    lib = FmmPlan(s, s, kappa, eps, precision="mixed", max_rhs=2, **kw)
    two = run_apply(lib, q)
    one = run_apply(lib, q[:, 0])
    assert rel(one, two[:, 0]) <= 1e-6
    w = torch.as_tensor(q, device="cuda")
    adj2 = lib.apply_adjoint(w).cpu().numpy()
    adj1 = lib.apply_adjoint(w[:, 0].contiguous()).cpu().numpy()
    assert rel(adj1, adj2[:, 0]) <= 1e-6
    assert rel(one, direct.direct(s, s, q[:, 0], kappa)) <= eps


def test_double_float_leaf_multi_rhs():
    """Double-float leaf level (S2M / L2T on the float32 pipe) with several right-hand
    sides: the kernels evaluate each plane wave once for a group of four RHS.  Column 1
    of a three-RHS apply must match a one-RHS apply (which also takes the symmetric
    near field) to float32 near-field round-off, the three-RHS apply must match the
    float64 policy to eps, and the adjoint must satisfy the dot-product identity."""
    import torch
    x = wl.sphere(20000, wl.rng(15))
    g = wl.rng(15, salt=1)
    q = wl.charges(len(x), 3, g)
    lib = FmmPlan(x, x, 64.0, 1e-6, precision="mixed", max_rhs=3)
    info = lib.info()
    assert info["levels"][info["lf"]]["precision"] == "df"
    three = run_apply(lib, q)
    one = run_apply(lib, q[:, 1])
    assert rel(one, three[:, 1]) <= 1e-6
    ref = run_apply(FmmPlan(x, x, 64.0, 1e-6, precision="fp64", max_rhs=3), q)
    assert rel(three, ref) <= 1e-6
    w = wl.charges(len(x), 3, g)
    aw = lib.apply_adjoint(torch.as_tensor(w, device="cuda")).cpu().numpy()
    lhs = np.vdot(w, three)                          # <w, A q>
    rhs = np.vdot(aw, q)                             # <A^H w, q>
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)


@pytest.mark.parametrize("nrhs", [9, 40])
def test_tensor_core_near_field(nrhs):
    """From 8 right-hand sides the float32 near field runs as a tensor-core GEMM form
    (mma.sync TF32, 3xTF32 split products).  With one box (no far field) the apply is the
    near field alone: it must match the float64 direct sum to float32 accuracy, apply and
    adjoint; R = 9 and 40 cover ragged passes of 32 RHS, ragged source tiles of 32 and a
    coincident pair.  Each column must also match the one-RHS scalar kernel."""
    import torch
    g = wl.rng(17, salt=nrhs)
    x = wl.cube(1500, g)
    x[10] = x[3]
    q = wl.charges(len(x), nrhs, g)
    lib = FmmPlan(x, x, 25.0, 1e-5, precision="mixed", max_leaf=4096, max_rhs=nrhs)
    assert lib.info()["near_precision"] == "fp32" and lib.info()["lf"] < 2
    got = run_apply(lib, q)
    want = direct.direct(x, x, q, 25.0)
    assert rel(got, want) <= 1e-6
    for r in (0, nrhs - 1):
        assert rel(run_apply(lib, q[:, r]), got[:, r]) <= 1e-6
    w = wl.charges(len(x), nrhs, g)
    adj = lib.apply_adjoint(torch.as_tensor(w, device="cuda")).cpu().numpy()
    assert rel(adj, direct.direct_adjoint(x, x, w, 25.0)) <= 1e-6


@pytest.mark.parametrize("kind", ["cube", "two_spheres"])
def test_two_buffer_boxes(kind):
    """Two buffer boxes (Section 3.3.3, |r0| >= 3 a_l; 5^3 neighbour lists, transfer vectors
    over [-5, 5]^3): float64 apply element-wise against the oracle FMM with the same option,
    mixed apply and adjoint within eps of the direct sums."""
    import torch
    g = wl.rng(130)
    if kind == "cube":
        s = t = wl.cube(2500, g)
        kappa, eps, kw = 70.0, 1e-6, dict(depth=3, root=(0, 0, 0, 1.0), buffer=2)
    else:
        s = wl.sphere(3000, g)
        t = wl.sphere(2000, g, radius=1.5)
        kappa, eps, kw = 16.0, 1e-6, dict(max_leaf=16, buffer=2)
    q = wl.charges(len(s), 0, wl.rng(131))
    lib = FmmPlan(s, t, kappa, eps, precision="fp64", **kw)
    orc = ofmm.Plan(s, t, kappa, eps, precision="fp64", **kw)
    assert lib.info()["lf"] == orc.lf >= 2 and lib.info()["buffer"] == 2
    got = run_apply(lib, q)
    check_fp64_parity(got, ofmm.apply(orc, q), orc, f"{kind}_buffer2")
    want = direct.direct(s, t, q, kappa)
    assert rel(got, want) <= eps
    mixed = FmmPlan(s, t, kappa, eps, precision="mixed", **kw)
    assert rel(run_apply(mixed, q, "c64"), want) <= eps
    w = wl.charges(len(t), 0, wl.rng(132))
    adj = mixed.apply_adjoint(torch.as_tensor(w, device="cuda")).cpu().numpy()
    assert rel(adj, direct.direct_adjoint(s, t, w, kappa)) <= eps
