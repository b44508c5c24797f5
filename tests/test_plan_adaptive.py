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
    assert len(set(orc.tree.leaf_level.tolist())) >= 2
    assert_same_plan(lib, orc)


def _covered_once(tr, max_targets=150):
    """Every (target leaf, source leaf) pair holding points is covered exactly once: directly or
    by M2L at one level of the two ancestor chains (target leaves on a strided sample of about
    max_targets, every source leaf)."""
    where = [{tuple(int(c) for c in L['idx'][i]): i for i in range(len(L['key']))} for L in tr.levels]
    anc = []
    for l, b in zip(tr.leaf_level, tr.leaf_box):
        i = tr.levels[l]['idx'][b]
        anc.append({m: where[m][tuple(int(c) for c in (i >> (l - m)))] for m in range(2, int(l) + 1)})
    nl = len(tr.leaf_level)
    for a in range(0, nl, max(1, nl // max_targets)):
        near = set(tr.nlist[a].tolist())
        for c in range(nl):
            if tr.tgt_count[a] == 0 or tr.src_count[c] == 0:
                continue
            m = min(int(tr.leaf_level[a]), int(tr.leaf_level[c]))
            m2l = sum(anc[c][l] in set(tr.ilist[l][anc[a][l]].tolist()) for l in range(2, m + 1))
            assert (c in near) + m2l == 1, (a, c)


def _line(n, g):
    x = np.zeros((n, 3))
    x[:, 0] = g.random(n)
    return x


EDGES = {
    # name: (sources, targets, kappa, eps, buffer, max_leaf)
    "coincident": (lambda g: (np.full((300, 3), 0.25), np.full((300, 3), 0.25)), 30.0, 1e-5, 1, 16),
    "one_point": (lambda g: (np.array([[0.1, 0.2, 0.3]]), np.array([[0.1, 0.2, 0.3]])), 30.0, 1e-5, 1, 16),
    "disjoint_corners": (lambda g: (0.1 * g.random((1500, 3)), 0.9 + 0.1 * g.random((1200, 3))), 80.0, 1e-5, 2, 16),
    "line": (lambda g: (_line(2000, g), _line(2000, g)), 60.0, 1e-5, 1, 8),
    "cluster_max_leaf_1": (lambda g: (np.concatenate([g.random((200, 3)), 0.5 + 0.01 * g.random((300, 3))]),) * 2,
                           40.0, 1e-4, 2, 1),
}


@pytest.mark.parametrize("name", sorted(EDGES))
def test_adaptive_edge_cases(name):
    make, kappa, eps, buffer, max_leaf = EDGES[name]
    s, t = make(wl.rng(83, salt=sorted(EDGES).index(name)))
    lib = FmmPlan(s, t, kappa, eps, precision="mixed", max_leaf=max_leaf, buffer=buffer, device=-1, adaptive=True)
    orc = ofmm.Plan(s, t, kappa, eps, precision="mixed", max_leaf=max_leaf, buffer=buffer, adaptive=True)
    assert_same_plan(lib, orc)
    tr = orc.tree
    assert tr.src_count.sum() == len(s) and tr.tgt_count.sum() == len(t)
    _covered_once(tr)


def assert_same_plan(lib, orc, ilist_sample=250):
    """Library host plan and oracle plan agree bit for bit (tree, leaves, near lists, plan
    integers; interaction lists of every box up to ilist_sample per level, else a strided
    sample)."""
    tr = orc.tree
    inf = lib.info()
    assert inf["adaptive"] and inf["lf"] == orc.lf == tr.depth and inf["occupancy_depth"] == orc.occupancy_depth
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
        n = len(tr.levels[l]['key'])
        assert len(io) == n + 1
        for a in range(0, n, max(1, n // ilist_sample)):
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


def _random_cloud(g):
    """Uniform background plus one to four dense cubes of random size and place."""
    parts = [g.random((int(g.integers(0, 400)), 3))]
    for _ in range(int(g.integers(1, 5))):
        c, h = g.uniform(0.05, 0.95, 3), g.uniform(0.005, 0.2)
        parts.append(np.clip(c + h * (g.random((int(g.integers(20, 600)), 3)) - 0.5), 0.0, 1.0))
    return np.concatenate(parts)


@pytest.mark.parametrize("seed", range(16))
def test_random_adaptive_plans(seed):
    """Seeded random clouds, max_leaf, buffer, depth and point-set pairings: the library's adaptive
    host plan equals the oracle's bit for bit and covers every leaf pair exactly once."""
    g = wl.rng(84, salt=seed)
    s = _random_cloud(g)
    t = s if g.random() < 0.6 else _random_cloud(g)
    max_leaf = int(g.integers(1, 48))
    buffer = int(g.integers(1, 3))
    depth = int(g.integers(2, 7))
    kappa = float(g.uniform(5.0, 80.0))
    lib = FmmPlan(s, t, kappa, 1e-4, precision="mixed", max_leaf=max_leaf, buffer=buffer, depth=depth,
                  root=(0, 0, 0, 1.0), device=-1, adaptive=True)
    orc = ofmm.Plan(s, t, kappa, 1e-4, precision="mixed", max_leaf=max_leaf, buffer=buffer, depth=depth,
                    root=(0, 0, 0, 1.0), adaptive=True)
    assert_same_plan(lib, orc, ilist_sample=40)
    _covered_once(orc.tree, max_targets=60)
