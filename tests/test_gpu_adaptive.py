"""GPU applies on adaptive trees (HFMM_FLAG_ADAPTIVE): leaves on several levels.

* float64 apply against the oracle's adaptive FMM element-wise at the float64 parity bound
  (same tree, lists and plan integers: the host plans are bit-exact, checked on the CPU);
* mixed applies within eps of the float64 direct sum: 1 right-hand side (the symmetric
  float32 near field), 3 (one-way float32), 20 (tcgen05 near field), a double-float near
  field (eps 1e-7), different sources and targets, and the plan-shape tuner (buffer = 0);
* adjoint: dot-product identity with the forward apply and the direct-sum adjoint;
* position gradient against the direct-sum gradient.
"""
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


def _clustered(n_spread, n_dense, g, side=0.05, centre=(0.7, 0.3, 0.6)):
    """Uniform points in the unit cube plus a dense small cube."""
    a = g.random((n_spread, 3))
    b = np.asarray(centre) + side * (g.random((n_dense, 3)) - 0.5)
    return np.concatenate([a, b])


def _levels(info):
    return {l: n for l, n in enumerate(info["level_nleaf"]) if n}


@pytest.mark.parametrize("buffer,kappa,eps", [(1, 60.0, 1e-6), (2, 20.0, 1e-6)])
def test_fp64_matches_oracle_adaptive_fmm(buffer, kappa, eps):
    g = wl.rng(90, salt=buffer)
    x = _clustered(2000, 3000, g, side=0.2)
    q = wl.charges(len(x), 2, g)
    kw = dict(max_leaf=48, buffer=buffer)
    plan = FmmPlan(x, x, kappa, eps, precision="fp64", max_rhs=2, adaptive=True, **kw)
    info = plan.info()
    assert info["adaptive"] and len(_levels(info)) >= 2, info["level_nleaf"]
    got = run_apply(plan, q)
    orc = ofmm.Plan(x, x, kappa, eps, precision="fp64", adaptive=True, **kw)
    assert orc.lf == info["lf"] and len(orc.tree.leaf_level) == info["nleaf"]
    want = ofmm.apply(orc, q)
    print(f"adaptive fp64 b={buffer}: leaves per level {_levels(info)}")
    check_fp64_parity(got, want, orc, f"adaptive b={buffer}")
    assert rel(got, direct.direct(x, x, q, kappa)) <= eps


CASES = {
    # name: (cloud, kappa, eps, nrhs, buffer, max_leaf, same points)
    "sym_r1": ("cube+cluster", 80.0, 1e-5, 1, 1, 48, True),
    "r3": ("cube+cluster", 80.0, 1e-5, 3, 2, 32, True),
    "tc5_r20": ("cube+cluster", 60.0, 1e-5, 20, 1, 64, True),
    "df_near": ("sphere+cluster", 50.0, 1e-7, 1, 2, 32, True),
    "src_tgt": ("cube+cluster", 60.0, 1e-6, 3, 1, 32, False),
    "tuned": ("clusters", 40.0, 1e-4, 1, 0, 64, True),
}


def _cloud(name, g):
    kind = CASES[name][0]
    if kind == "cube+cluster":
        x = _clustered(2000, 22000, g, side=0.3)
    elif kind == "clusters":
        x = wl.clusters(80000, g)
    else:
        x = np.concatenate([0.5 + 0.5 * wl.sphere(15000, g),
                            np.array([0.45, 0.5, 0.55]) + 0.04 * (g.random((10000, 3)) - 0.5)])
    if CASES[name][6]:
        return x, x
    return x, _clustered(1500, 12000, g, side=0.3, centre=(0.3, 0.6, 0.4))


@pytest.mark.parametrize("name", sorted(CASES))
def test_mixed_within_eps_of_direct_sum(name):
    _, kappa, eps, nrhs, buffer, max_leaf, _ = CASES[name]
    g = wl.rng(91, salt=sorted(CASES).index(name))
    s, t = _cloud(name, g)
    q = wl.charges(len(s), nrhs, g)
    plan = FmmPlan(s, t, kappa, eps, precision="mixed", max_rhs=nrhs, max_leaf=max_leaf, buffer=buffer,
                   adaptive=True)
    info = plan.info()
    got = run_apply(plan, q)
    idx = np.sort(g.choice(len(t), 400, replace=False))
    err = rel(got[idx], direct.direct(s, t[idx], q, kappa))
    print(f"adaptive {name}: lf={info['lf']} buffer={info['buffer']} leaves {_levels(info)} "
          f"near={info['near_precision']} sym={info['near_symmetric']} mma_tiles={info['near_mma_tiles']} "
          f"rel err {err:.2e}")
    assert len(_levels(info)) >= 2
    if name == "tc5_r20":
        assert info["near_mma_tiles"] > 0
    if name == "sym_r1":
        assert info["near_symmetric"]
    assert err <= eps, (name, err)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adjoint_on_adaptive_tree(precision):
    import torch
    g = wl.rng(92)
    s = _clustered(1500, 4000, g, side=0.2)
    t = _clustered(1000, 3000, g, side=0.2, centre=(0.3, 0.6, 0.4))
    kappa, eps = 60.0, 1e-6
    kw = dict(max_leaf=32, buffer=1)
    plan = FmmPlan(s, t, kappa, eps, precision=precision, max_rhs=2, adaptive=True, **kw)
    assert len(_levels(plan.info())) >= 2
    x = wl.charges(len(s), 2, g)
    y = wl.charges(len(t), 2, g)
    ax = run_apply(plan, x)
    ahy = plan.apply_adjoint(torch.as_tensor(y, device="cuda")).cpu().numpy()
    lhs, rhs = np.vdot(y, ax), np.vdot(ahy, x)
    scale = np.linalg.norm(ax) * np.linalg.norm(y)
    tol = fp64_parity_tol(ofmm.Plan(s, t, kappa, eps, precision="fp64", adaptive=True, **kw)) \
        if precision == "fp64" else 1e-6
    assert abs(lhs - rhs) <= tol * scale, abs(lhs - rhs) / scale
    assert rel(ahy, direct.direct_adjoint(s, t, y, kappa)) <= eps


def test_gradient_on_adaptive_tree():
    import torch
    g = wl.rng(93)
    s = _clustered(1500, 3000, g, side=0.2)
    t = _clustered(1000, 2000, g, side=0.2, centre=(0.3, 0.6, 0.4))
    kappa, eps = 60.0, 1e-6
    q = wl.charges(len(s), 0, g)
    qstar = q + 0.01 * wl.charges(len(s), 0, g)
    plan = FmmPlan(s, t, kappa, eps, precision="fp64", max_leaf=32, adaptive=True)
    assert len(_levels(plan.info())) >= 2
    phistar = direct.direct(s, t, qstar, kappa)
    resid = run_apply(plan, q) - phistar
    grad = plan.grad_sources(torch.as_tensor(q, device="cuda"),
                             torch.as_tensor(2.0 * resid, device="cuda")).cpu().numpy()
    want = direct.direct_grad_sources(s, t, q, direct.direct(s, t, q, kappa) - phistar, kappa)
    assert rel(grad, want) <= 20 * eps
