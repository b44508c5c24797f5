"""Pins of the oracle's octree and lists against brute force (Section 2 definitions)."""
import itertools

import numpy as np
import pytest

from oracle import tree as tr


def _brute(points_s, points_t, corner, side, depth):
    levels = []
    for l in range(depth + 1):
        nb = 2 ** l
        boxes = set()
        for p in np.concatenate([points_s, points_t]):
            i = np.clip(np.floor((p - corner) * (nb / side)), 0, nb - 1).astype(int)
            boxes.add(tuple(i))
        levels.append(boxes)
    return levels


def _cheb(a, b):
    return max(abs(x - y) for x, y in zip(a, b))


@pytest.mark.parametrize("seed,n,depth,buffer", [(0, 300, 3, 1), (1, 500, 4, 1), (2, 60, 2, 1),
                                                 (3, 400, 3, 2), (4, 700, 4, 2)])
def test_lists_match_definitions(seed, n, depth, buffer):
    """Interaction list = boxes farther than `buffer` (Chebyshev) whose parents are within
    `buffer` of the parent (Section 2, with b buffer boxes, Section 3.3.3); neighbour list =
    boxes within `buffer`.  |I| <= (2b+1)^3 * 8 - (2b+1)^3 (189 for b = 1, 875 for b = 2)."""
    rng = np.random.default_rng(seed)
    src = rng.random((n, 3)) ** 2          # clustered towards a corner
    tgt = rng.random((n // 2, 3))
    t = tr.Tree(src, tgt, depth, buffer=buffer)
    brute = _brute(src, tgt, t.corner, t.side, depth)
    span = 2 * buffer + 1
    for l in range(depth + 1):
        got = {tuple(int(c) for c in i) for i in t.levels[l]['idx']}
        assert got == brute[l]
    for l in range(2, depth + 1):
        idx = [tuple(int(c) for c in i) for i in t.levels[l]['idx']]
        for a, ia in enumerate(idx):
            want = sorted(b for b, ib in enumerate(idx)
                          if _cheb(ia, ib) > buffer
                          and _cheb([x >> 1 for x in ia], [x >> 1 for x in ib]) <= buffer)
            assert sorted(t.ilist[l][a].tolist()) == want
            assert len(want) <= span ** 3 * 8 - span ** 3
            for b, v in zip(t.ilist[l][a], t.vlist[l][a]):
                d = np.array(idx[b]) - np.array(ia)
                assert buffer + 1 <= np.max(np.abs(d)) <= span
                assert v == tr.transfer_index(d, buffer)
                assert np.array_equal(tr.transfer_offset(v, buffer), d)
            keys = t.levels[l]['key'][t.ilist[l][a]]
            assert np.all(np.diff(keys) > 0)
        # symmetry: b in I(a) <=> a in I(b)
        for a in range(len(idx)):
            for b in t.ilist[l][a]:
                assert a in t.ilist[l][b]
    idx = [tuple(int(c) for c in i) for i in t.levels[depth]['idx']]
    for a, ia in enumerate(idx):
        assert sorted(t.nlist[a].tolist()) == sorted(b for b, ib in enumerate(idx) if _cheb(ia, ib) <= buffer)


def test_points_in_their_boxes_and_parents():
    rng = np.random.default_rng(4)
    src = rng.standard_normal((400, 3))
    t = tr.Tree(src, src, 3)
    lev = t.levels[3]
    h = t.side / 8
    ys = src[t.src_perm]
    for b in range(len(lev['key'])):
        s0, sc = t.src_start[b], t.src_count[b]
        d = np.abs(ys[s0:s0 + sc] - lev['center'][b])
        assert np.all(d <= h / 2 * (1 + 1e-12))
    assert t.src_count.sum() == 400 and t.tgt_count.sum() == 400
    for l in range(1, 4):
        par = t.levels[l - 1]
        ch = t.levels[l]
        assert np.all(par['idx'][ch['parent']] == ch['idx'] >> 1)
    # points sorted by key, ties by original index
    keys = tr.morton_key(tr.box_index(ys, t.corner, t.side, 3), 3)
    assert np.all(np.diff(keys) >= 0)
    same = np.diff(keys) == 0
    assert np.all(np.diff(t.src_perm)[same] > 0)


@pytest.mark.parametrize("buffer,nvec,ncanon", [(1, 316, 34), (2, 1206, 108)])
def test_transfer_vectors_and_canonical(buffer, nvec, ncanon):
    """Offsets of interaction-list boxes: [-(2b+1), 2b+1]^3 without [-b, b]^3 (316 for one
    buffer box, Section 3.3.2); up to the reflections x -> -x, y -> -y, z -> -z and x <-> y,
    34 (Figure SemiOctant) or 108 canonical ones with x >= y >= 0, z >= 0."""
    D = 2 * buffer + 1
    vecs = [d for d in itertools.product(range(-D, D + 1), repeat=3) if max(map(abs, d)) > buffer]
    assert len(vecs) == nvec
    canon = {(max(abs(d[0]), abs(d[1])), min(abs(d[0]), abs(d[1])), abs(d[2])) for d in vecs}
    assert len(canon) == ncanon
    idx = {tr.transfer_index(d, buffer) for d in vecs}
    assert len(idx) == nvec and max(idx) < (2 * D + 1) ** 3


def test_root_cube_and_depth():
    rng = np.random.default_rng(9)
    p = rng.random((1000, 3)) * [2.0, 1.0, 0.5] + 3.0
    c, s = tr.root_cube(p)
    assert s == pytest.approx(np.max(p.max(0) - p.min(0)))
    assert np.all(p >= c) and np.all(p <= c + s)
    d = tr.occupancy_depth(p, p, c, s, 64)
    assert tr.max_occupancy(p, p, c, s, d) <= 64 < tr.max_occupancy(p, p, c, s, d - 1)
