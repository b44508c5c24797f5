"""The library's adaptive host plan (HFMM_FLAG_ADAPTIVE) against the oracle's adaptive tree,
bit for bit (CPU only; host-only plans): permutations, the boxes of every level with their
parents, the leaves (level, position, point ranges) in Morton order, the near lists, the
interaction lists and transfer vectors, and the plan integers.  Clouds with strong density
contrast put leaves on two to four levels.
"""
import zlib

import numpy as np
import pytest

from oracle import fmm as ofmm
from paper_0911_4114_gb300 import FmmPlan, workloads as wl


def _cloud(kind, g):
    if kind == "cube_and_cluster":
        x = np.concatenate([g.random((1500, 3)), np.array([0.7, 0.3, 0.6]) + 0.04 * (g.random((1500, 3)) - 0.5)])
        return x, x
    if kind == "sphere_and_cluster":
        s = wl.sphere(2500, g)
        c = np.array([0.2, -0.1, 0.3]) + 0.05 * (g.random((1500, 3)) - 0.5)
        x = np.concatenate([s, c])
        return x, x
    # different sources and targets: a clustered source cloud, spread targets
    x = np.concatenate([g.random((800, 3)), np.array([0.3, 0.3, 0.3]) + 0.03 * (g.random((1200, 3)) - 0.5)])
    return x, g.random((1500, 3))


CASES = [
    ("cube_and_cluster", 60.0, 1e-4, 1, 32),
    ("cube_and_cluster", 20.0, 1e-6, 2, 8),
    ("sphere_and_cluster", 80.0, 1e-6, 1, 32),
    ("sources_clustered", 40.0, 1e-5, 2, 16),
]


@pytest.mark.parametrize("kind,kappa,eps,buffer,max_leaf", CASES)
def test_adaptive_host_plan_bit_exact(kind, kappa, eps, buffer, max_leaf):
    g = wl.rng(81, salt=zlib.crc32(f"{kind}/{buffer}/{max_leaf}".encode()) % 1000)
    s, t = _cloud(kind, g)
    lib = FmmPlan(s, t, kappa, eps, precision="mixed", max_leaf=max_leaf, buffer=buffer, device=-1, adaptive=True)
    orc = ofmm.Plan(s, t, kappa, eps, precision="mixed", max_leaf=max_leaf, buffer=buffer, adaptive=True)
    tr = orc.tree
    inf = lib.info()
    assert inf["adaptive"] and inf["lf"] == orc.lf == tr.depth and inf["occupancy_depth"] == orc.occupancy_depth
    assert len(set(tr.leaf_level.tolist())) >= 2
    assert np.array_equal(lib.debug_get("SRC_PERM"), tr.src_perm)
    assert np.array_equal(lib.debug_get("TGT_PERM"), tr.tgt_perm)
    for l in range(tr.depth + 1):
        assert np.array_equal(lib.debug_get("BOX_IDX", l), tr.levels[l]['idx']), l
        if l > 0:
            assert np.array_equal(lib.debug_get("BOX_PARENT", l), tr.levels[l]['parent']), l
        assert inf["level_nleaf"][l] == int(tr.levels[l]['leaf'].sum())
    lb = lib.debug_get("LEAF_BOX")
    assert inf["nleaf"] == len(tr.leaf_level)
    assert np.array_equal(lb[:, 0], tr.leaf_level) and np.array_equal(lb[:, 1], tr.leaf_box)
    ls, lt = lib.debug_get("LEAF_SRC"), lib.debug_get("LEAF_TGT")
    assert np.array_equal(ls[:, 0], tr.src_start) and np.array_equal(ls[:, 1], tr.src_count)
    assert np.array_equal(lt[:, 0], tr.tgt_start) and np.array_equal(lt[:, 1], tr.tgt_count)
    off, idx = lib.debug_get("NLIST_OFF"), lib.debug_get("NLIST_IDX")
    pairs = 0
    for a in range(len(tr.leaf_level)):
        assert np.array_equal(idx[off[a]:off[a + 1]], tr.nlist[a]), a
        pairs += int(tr.tgt_count[a]) * int(tr.src_count[tr.nlist[a]].sum())
    assert inf["p2p_pairs"] == pairs
    for l in range(2, tr.depth + 1):
        io, ii, iv = lib.debug_get("ILIST_OFF", l), lib.debug_get("ILIST_IDX", l), lib.debug_get("ILIST_V", l)
        for a in range(len(tr.levels[l]['key'])):
            assert np.array_equal(ii[io[a]:io[a + 1]], tr.ilist[l][a]), (l, a)
            assert np.array_equal(iv[io[a]:io[a + 1]], tr.vlist[l][a]), (l, a)
        lv = inf["levels"][l]
        assert lv["ell"] == orc.levels[l].ell and lv["ntheta"] == orc.levels[l].ntheta
        assert np.array_equal(lib.debug_get("NPHI", l), orc.levels[l].quad.nphi)
        assert lv["precision"] == orc.level_precision[l]


def test_uniform_plan_reports_its_leaves():
    g = wl.rng(82)
    x = g.random((3000, 3))
    lib = FmmPlan(x, x, 40.0, 1e-5, precision="mixed", device=-1)
    inf = lib.info()
    lf = inf["lf"]
    assert not inf["adaptive"] and inf["nleaf"] == inf["nbox"][lf]
    assert inf["level_nleaf"] == [0] * lf + [inf["nbox"][lf]]
    lb = lib.debug_get("LEAF_BOX")
    assert np.all(lb[:, 0] == lf) and np.array_equal(lb[:, 1], np.arange(inf["nbox"][lf]))
