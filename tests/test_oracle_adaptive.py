"""Pins of the oracle's adaptive octree (leaves on several levels) and its FMM.

* every (target leaf, source leaf) pair is covered exactly once: either directly (the
  source leaf is in the target leaf's near list) or by M2L at exactly one level l, where
  the source leaf's level-l ancestor is in the interaction list of the target leaf's
  level-l ancestor -- counted by walking both ancestor chains, independently of how the
  lists were built;
* the leaves partition the points and each point lies inside its leaf's cube;
* the split rule: a box has children iff it is above the depth and above level 2, holds
  more than max_leaf sources or targets, or holds a point while the other cubes of its level
  within Chebyshev distance b hold more than (2b+1)^3 max_leaf sources or targets (counted
  here from the point coordinates);
* max_leaf = 0 splits every box: the tree, lists and ranges equal the uniform tree's;
* the adaptive FMM on strongly clustered clouds matches the float64 direct sum within eps.
"""
import numpy as np
import pytest

from oracle import direct, fmm
from oracle.tree import Tree
from paper_0911_4114_gb300 import workloads as wl


def _clustered(n_spread, n_dense, g, side=0.04, centre=(0.7, 0.3, 0.6)):
    """Uniform points in the unit cube plus a dense small cube: leaves on several levels."""
    a = g.random((n_spread, 3))
    b = np.asarray(centre) + side * (g.random((n_dense, 3)) - 0.5)
    return np.concatenate([a, b])


def _ancestor_pos(t, l_leaf, idx, l):
    """Position at level l of the ancestor of a box of level l_leaf with coordinates idx."""
    anc = np.asarray(idx) >> (l_leaf - l)
    where = {tuple(int(c) for c in t.levels[l]['idx'][i]): i for i in range(len(t.levels[l]['key']))}
    return where[tuple(int(c) for c in anc)]


@pytest.mark.parametrize("buffer", [1, 2])
@pytest.mark.parametrize("max_leaf", [4, 12])
def test_every_leaf_pair_covered_exactly_once(buffer, max_leaf):
    g = wl.rng(71, salt=buffer * 100 + max_leaf)
    x = _clustered(150, 150, g)
    y = _clustered(120, 100, g, centre=(0.25, 0.7, 0.4))
    t = Tree(x, y, 6, buffer=buffer, max_leaf=max_leaf)
    assert len(set(t.leaf_level.tolist())) >= 3          # leaves on several levels
    nleaf = len(t.leaf_level)
    idx = [t.levels[l]['idx'][b] for l, b in zip(t.leaf_level, t.leaf_box)]
    anc = [{l: _ancestor_pos(t, int(t.leaf_level[a]), idx[a], l) for l in range(2, int(t.leaf_level[a]) + 1)}
           for a in range(nleaf)]
    ilists = {l: [set(t.ilist[l][a].tolist()) for a in range(len(t.levels[l]['key']))]
              for l in range(2, t.depth + 1)}
    for a in range(nleaf):
        near = set(t.nlist[a].tolist())
        for c in range(nleaf):
            m = min(int(t.leaf_level[a]), int(t.leaf_level[c]))
            m2l = sum(anc[c][l] in ilists[l][anc[a][l]] for l in range(2, m + 1))
            assert (c in near) + m2l == 1, (a, c, c in near, m2l)


def test_leaves_partition_points_and_follow_the_split_rule():
    g = wl.rng(72)
    x = _clustered(300, 300, g)
    max_leaf = 10
    t = Tree(x, x, 7, buffer=1, max_leaf=max_leaf)
    # ranges tile [0, n) in leaf order, each point inside its leaf's cube
    for start, count in ((t.src_start, t.src_count), (t.tgt_start, t.tgt_count)):
        assert start[0] == 0 and np.all(start[1:] == start[:-1] + count[:-1])
        assert start[-1] + count[-1] == len(x)
    xs = x[t.src_perm]
    for a, (l, b) in enumerate(zip(t.leaf_level, t.leaf_box)):
        h = t.side / 2.0 ** l
        lo = t.corner + t.levels[l]['idx'][b] * h
        p = xs[t.src_start[a]:t.src_start[a] + t.src_count[a]]
        assert np.all(p >= lo - 1e-12) and np.all(p <= lo + h + 1e-12)
    lim = 27 * max_leaf
    crowd_only = 0          # boxes split only because they are crowded
    for l, L in enumerate(t.levels):
        big = (L['src_count'] > max_leaf) | (L['tgt_count'] > max_leaf)
        # points in the other cubes within Chebyshev distance 1, from the coordinates
        pc = np.clip(np.floor((x - t.corner) * (2 ** l / t.side)), 0, 2 ** l - 1).astype(np.int64)
        crowd = np.zeros(len(L['key']), dtype=bool)
        for b in range(len(L['key'])):
            cheb = np.max(np.abs(pc - L['idx'][b]), axis=1)
            around = int(np.count_nonzero((cheb >= 1) & (cheb <= 1)))
            crowd[b] = L['src_count'][b] + L['tgt_count'][b] > 0 and around > lim
        assert np.array_equal(L['split'], (l < t.depth) & ((l < 2) | big | crowd)), l
        if 2 <= l < t.depth:
            crowd_only += int(np.count_nonzero(crowd & ~big))
        if l > 0:   # boxes exist only below split boxes
            assert np.all(t.levels[l - 1]['split'][L['parent']])
            assert np.all(L['src_count'] + L['tgt_count'] > 0)
    assert crowd_only > 0


def test_max_leaf_zero_is_the_uniform_tree():
    g = wl.rng(73)
    x = _clustered(200, 200, g)
    y = g.random((150, 3))
    u = Tree(x, y, 5, buffer=2)
    a = Tree(x, y, 5, buffer=2, max_leaf=0)
    assert np.array_equal(u.src_perm, a.src_perm) and np.array_equal(u.tgt_perm, a.tgt_perm)
    for l in range(6):
        assert np.array_equal(u.levels[l]['key'], a.levels[l]['key'])
    assert np.all(a.leaf_level == 5) and np.array_equal(a.leaf_box, np.arange(len(u.levels[5]['key'])))
    for f in ('src_start', 'src_count', 'tgt_start', 'tgt_count'):
        assert np.array_equal(getattr(u, f), getattr(a, f))
    # lists on a strided sample of about 150 boxes per level
    n = len(u.nlist)
    for b in range(0, n, max(1, n // 150)):
        assert np.array_equal(u.nlist[b], a.nlist[b])
    for l in range(2, 6):
        n = len(u.levels[l]['key'])
        for b in range(0, n, max(1, n // 150)):
            assert np.array_equal(u.ilist[l][b], a.ilist[l][b])
            assert np.array_equal(u.vlist[l][b], a.vlist[l][b])


@pytest.mark.parametrize("buffer,kappa,eps", [(1, 60.0, 1e-4), (1, 100.0, 1e-6), (2, 12.0, 1e-6), (2, 20.0, 1e-4)])
def test_adaptive_fmm_matches_direct_sum(buffer, kappa, eps):
    g = wl.rng(74, salt=buffer)
    x = _clustered(700, 900, g, side=0.1)
    q = g.standard_normal(len(x)) + 1j * g.standard_normal(len(x))
    plan = fmm.Plan(x, x, kappa, eps, max_leaf=16, buffer=buffer, adaptive=True)
    t = plan.tree
    assert plan.lf >= 3 and len(set(t.leaf_level.tolist())) >= 2
    phi = fmm.apply(plan, q)
    want = direct.direct(x, x, q, kappa)
    err = np.linalg.norm(phi - want) / np.linalg.norm(want)
    assert err <= eps, err


@pytest.mark.parametrize("seed", range(7))
def test_direct_work_of_a_leaf_is_bounded(seed):
    """The crowded-box rule bounds what a leaf above the depth sums directly: the leaves under its
    level-l neighbours hold at most (2b+1)^3 max_leaf + max_leaf sources (itself and the other
    cubes, which are not crowded), and each coarser level m < l adds at most (2b+1)^3 - 1 leaves of
    at most max_leaf sources (leaves neighbouring the level-m ancestor)."""
    g = wl.rng(75, salt=seed)
    if seed == 6:
        # a sparse background with a very dense small cube: without the rule, sparse leaves next to
        # the cube would sum all of its points directly
        x = np.concatenate([g.random((80, 3)), np.array([0.26, 0.26, 0.26]) + 0.02 * g.random((4000, 3))])
    else:
        parts = [g.random((int(g.integers(50, 400)), 3))]
        for _ in range(int(g.integers(1, 4))):
            c, h = g.uniform(0.1, 0.9, 3), g.uniform(0.01, 0.15)
            parts.append(np.clip(c + h * (g.random((int(g.integers(100, 800)), 3)) - 0.5), 0.0, 1.0))
        x = np.concatenate(parts)
    buffer, max_leaf = 1 + seed % 2, int(g.integers(2, 30))
    t = Tree(x, x, 6, root=(0, 0, 0, 1.0), buffer=buffer, max_leaf=max_leaf)
    span = (2 * buffer + 1) ** 3
    checked = 0
    for a in range(len(t.leaf_level)):
        l = int(t.leaf_level[a])
        if l == t.depth:
            continue
        direct_src = int(t.src_count[t.nlist[a]].sum())
        assert direct_src <= span * max_leaf + max_leaf + l * (span - 1) * max_leaf, (a, l, direct_src)
        checked += 1
    assert checked > 0
