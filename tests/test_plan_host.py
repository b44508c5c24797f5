"""The library's host planner against the oracle's (CPU only; host-only plans, no GPU).

Integer work (tree, lists, permutations, l, N_theta, N_phi, active levels, alpha and
precision choices) must agree bit for bit; the T^{s,LL} tables (the library computes
34 vectors and reflects them, the oracle computes every vector directly) must agree to
round-off.
"""
import zlib

import numpy as np
import pytest

from oracle import fmm as ofmm
from oracle import quadrature as oq
from paper_0911_4114_gb300 import FmmPlan

CASES = {
    "cube_low_freq": dict(n=1500, kind="cube", kappa=8 * np.pi, eps=1e-6, depth=3, root=(0, 0, 0, 1.0)),
    "cube_two_levels": dict(n=1200, kind="cube", kappa=60.0, eps=1e-6, depth=3, root=(0, 0, 0, 1.0)),
    "sphere_auto_depth": dict(n=3000, kind="sphere", kappa=24.0, eps=1e-5, depth=0, root=None, max_leaf=32),
    "two_spheres": dict(n=800, kind="two", kappa=12.0, eps=1e-6, depth=0, root=None, max_leaf=16),
    "sphere_tight_eps": dict(n=3000, kind="sphere", kappa=60.0, eps=1e-9, depth=0, root=None, max_leaf=16),
    # two buffer boxes (Section 3.3.3): 5^3 neighbour lists, offsets in [-5, 5]^3
    "cube_two_buffer": dict(n=2500, kind="cube", kappa=70.0, eps=1e-6, depth=3, root=(0, 0, 0, 1.0), buffer=2),
    "spheres_two_buffer": dict(n=1500, kind="two", kappa=16.0, eps=1e-6, depth=0, root=None, max_leaf=16,
                               buffer=2),
}


def _points(c, rng):
    n = c["n"]
    if c["kind"] == "cube":
        x = rng.random((n, 3))
        return x, x
    s = rng.standard_normal((n, 3))
    s /= np.linalg.norm(s, axis=1)[:, None]
    if c["kind"] == "sphere":
        return s, s
    t = rng.standard_normal((n // 2, 3))
    t *= 1.5 / np.linalg.norm(t, axis=1)[:, None]
    return s, t


@pytest.fixture(scope="module", params=sorted(CASES))
def pair(request):
    c = CASES[request.param]
    rng = np.random.default_rng(zlib.crc32(request.param.encode()))
    s, t = _points(c, rng)
    kw = dict(depth=c["depth"], root=c["root"], max_leaf=c.get("max_leaf", 64), buffer=c.get("buffer", 1))
    out = {}
    for prec in ("fp64", "mixed"):
        lib = FmmPlan(s, t, c["kappa"], c["eps"], precision=prec, device=-1, **kw)
        orc = ofmm.Plan(s, t, c["kappa"], c["eps"], precision=prec, **kw)
        out[prec] = (lib, orc)
    return request.param, out


def test_levels_and_quadrature_integers(pair):
    name, out = pair
    for prec, (lib, orc) in out.items():
        info = lib.info()
        assert info["lf"] == orc.lf, (name, prec)
        assert info["occupancy_depth"] == orc.occupancy_depth
        assert info["buffer"] == orc.buffer
        for l, lp in orc.levels.items():
            li = info["levels"][l]
            assert (li["ell"], li["ntheta"], li["K"]) == (lp.ell, lp.ntheta, lp.K), (name, prec, l)
            assert li["alpha"] == lp.alpha
            assert li["alpha"] in ofmm.alpha_ladder(orc.eps)
            assert orc.kappa * lp.a >= ofmm.min_ka(orc.buffer)   # one buffer box: about a wavelength or more
            assert li["precision"] == orc.level_precision[l]
            assert np.array_equal(lib.debug_get("NPHI", l), lp.nphi)
            assert li["round_est"] == pytest.approx(lp.rounding_estimate(
                ofmm.PRECISION_UNIT[orc.level_precision[l]]), rel=1e-9)


def test_tree_and_lists_bit_exact(pair):
    name, out = pair
    lib, orc = out["fp64"]
    t = orc.tree
    assert np.array_equal(lib.debug_get("SRC_PERM"), t.src_perm)
    assert np.array_equal(lib.debug_get("TGT_PERM"), t.tgt_perm)
    for l in range(t.depth + 1):
        assert np.array_equal(lib.debug_get("BOX_IDX", l), t.levels[l]["idx"])
        if l > 0:
            assert np.array_equal(lib.debug_get("BOX_PARENT", l), t.levels[l]["parent"])
    for l in range(2, t.depth + 1):
        off = lib.debug_get("ILIST_OFF", l)
        idx = lib.debug_get("ILIST_IDX", l)
        v = lib.debug_get("ILIST_V", l)
        for a in range(len(t.ilist[l])):
            assert np.array_equal(idx[off[a]:off[a + 1]], t.ilist[l][a])
            assert np.array_equal(v[off[a]:off[a + 1]], t.vlist[l][a])
    off = lib.debug_get("NLIST_OFF")
    idx = lib.debug_get("NLIST_IDX")
    for a in range(len(t.nlist)):
        assert np.array_equal(idx[off[a]:off[a + 1]], t.nlist[a])
    ls = lib.debug_get("LEAF_SRC")
    lt = lib.debug_get("LEAF_TGT")
    assert np.array_equal(ls[:, 1], t.src_count) and np.array_equal(lt[:, 1], t.tgt_count)
    nz = t.src_count > 0
    assert np.array_equal(ls[nz, 0], t.src_start[nz])


def test_transfer_tables(pair):
    name, out = pair
    lib, orc = out["fp64"]
    t = orc.tree
    for l in range(2, t.depth + 1):
        vs = sorted(set(np.concatenate(t.vlist[l]).tolist()))
        for v in vs[:: max(1, len(vs) // 12)]:
            a = lib.debug_get("TABLE", l, v)
            b = orc.table(l, v)
            scale = np.max(np.abs(b))
            est = orc.levels[l].rounding_estimate(oq.U_FP64)
            assert np.max(np.abs(a - b)) <= max(1e-11, 1e3 * est) * scale, (name, l, v)


def test_all_316_reflections_match_direct():
    rng = np.random.default_rng(0)
    x = rng.random((600, 3))
    lib = FmmPlan(x, x, 60.0, 1e-4, depth=2, root=(0, 0, 0, 1.0), device=-1)
    orc = ofmm.Plan(x, x, 60.0, 1e-4, depth=2, root=(0, 0, 0, 1.0))
    assert lib.info()["lf"] == 2
    lp = orc.levels[2]
    worst = 0.0
    for v in range(343):
        d = np.array([v // 49 - 3, (v // 7) % 7 - 3, v % 7 - 3])
        if np.max(np.abs(d)) < 2:
            with pytest.raises(KeyError):
                lib.debug_get("TABLE", 2, v)
            continue
        a = lib.debug_get("TABLE", 2, v)
        b = oq.tsll(lp.ell, 60.0, d * 0.25, lp.ntheta, lp.nphi)
        worst = max(worst, np.max(np.abs(a - b)) / np.max(np.abs(b)))
    assert worst < 1e-12


def test_near_field_policy_and_symmetry_flags():
    """Host plan properties that select kernels: the near-field arithmetic follows the
    precision policy and eps (mixed: float32 for eps >= 1e-6, double-float down to 1e-11,
    float64 below; float64 policy: float64); the symmetric near field is chosen exactly
    when the two point sets are equal (same values, not just the same multiset) and the
    near field is float32; self pairs are sum_b n_b^2 over leaf boxes."""
    rng = np.random.default_rng(zlib.crc32(b"near-policy"))
    x = rng.random((3000, 3))
    kw = dict(depth=3, root=(0, 0, 0, 1.0), device=-1)
    cases = [("mixed", 1e-5, "fp32"), ("mixed", 1e-6, "fp32"), ("mixed", 9.9e-7, "df"),
             ("mixed", 1e-11, "df"), ("mixed", 9e-12, "fp64"), ("fp64", 1e-5, "fp64")]
    for prec, eps, want in cases:
        info = FmmPlan(x, x, 20.0, eps, precision=prec, **kw).info()
        assert info["near_precision"] == want, (prec, eps)
        assert info["near_symmetric"] == (want == "fp32")
    perm = rng.permutation(len(x))
    assert not FmmPlan(x, x[perm], 20.0, 1e-5, precision="mixed", **kw).info()["near_symmetric"]
    assert FmmPlan(x, x.copy(), 20.0, 1e-5, precision="mixed", **kw).info()["near_symmetric"]
    lib = FmmPlan(x, x, 20.0, 1e-5, precision="mixed", **kw)
    t = ofmm.Plan(x, x, 20.0, 1e-5, precision="mixed", depth=3, root=(0, 0, 0, 1.0)).tree
    info = lib.info()
    assert info["p2p_self_pairs"] == int(np.sum(t.src_count.astype(np.int64) * t.tgt_count))
    assert 0 < info["p2p_self_pairs"] < info["p2p_pairs"]


def test_plan_independent_of_thread_count(tmp_path):
    """The planner's parallel loops (quadrature search, transfer tables, interaction lists)
    compute independent items: a plan built with one OpenMP thread must equal the default
    one bit for bit."""
    import os
    import pickle
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "dump.py"
    script.write_text(
        "import sys, pickle, numpy as np\n"
        f"sys.path.insert(0, {root!r})\n"
        "from paper_0911_4114_gb300 import FmmPlan\n"
        "x = np.random.default_rng(5).random((2000, 3))\n"
        "p = FmmPlan(x, x, 50.0, 1e-7, precision='mixed', depth=3, root=(0, 0, 0, 1.0), device=-1)\n"
        "out = {'lf': p.info()['lf'], 'perm': p.debug_get('SRC_PERM')}\n"
        "for l in range(2, out['lf'] + 1):\n"
        "    out[('nphi', l)] = p.debug_get('NPHI', l)\n"
        "    for v in (0 * 49 + 1 * 7 + 5, 5 * 49 + 3 * 7 + 0, 6 * 49 + 6 * 7 + 6, 1 * 49 + 6 * 7 + 3):\n"
        "        out[('T', l, v)] = p.debug_get('TABLE', l, v)\n"
        "pickle.dump(out, open(sys.argv[1], 'wb'))\n")
    res = {}
    for threads in ("1", "4"):
        f = tmp_path / f"plan{threads}.pkl"
        env = dict(os.environ, OMP_NUM_THREADS=threads)
        subprocess.run([sys.executable, str(script), str(f)], check=True, env=env)
        res[threads] = pickle.load(open(f, "rb"))
    a, b = res["1"], res["4"]
    assert a.keys() == b.keys() and a["lf"] >= 2
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_tuned_plan_equals_forced_plan():
    """buffer = 0: the plan-shape tuner picks the candidate (buffer, leaf level) of least
    predicted time, and the plan is exactly the plan with that buffer and depth = lf."""
    rng = np.random.default_rng(zlib.crc32(b"tuner"))
    x = rng.random((6000, 3))
    for kappa, eps in ((70.0, 1e-4), (24.0, 1e-6)):
        auto = FmmPlan(x, x, kappa, eps, precision="mixed", max_leaf=32, buffer=0, device=-1)
        ia = auto.info()
        assert ia["tuned"] and ia["lf"] >= 2
        assert ia["predicted_ms"][(ia["buffer"], ia["lf"])] == min(ia["predicted_ms"].values())
        forced = FmmPlan(x, x, kappa, eps, precision="mixed", buffer=ia["buffer"], depth=ia["lf"], device=-1)
        fi = forced.info()
        assert fi["lf"] == ia["lf"] and fi["levels"] == ia["levels"]
        for what in ("SRC_PERM", "NLIST_OFF", "NLIST_IDX"):
            assert np.array_equal(auto.debug_get(what), forced.debug_get(what))
        for l in range(2, ia["lf"] + 1):
            for what in ("BOX_IDX", "ILIST_OFF", "ILIST_IDX", "ILIST_V", "NPHI"):
                assert np.array_equal(auto.debug_get(what, l), forced.debug_get(what, l)), (what, l)
