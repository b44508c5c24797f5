"""Octree, interaction lists and neighbour lists (oracle; test infrastructure only).

Follows Section 2 of the paper (the FMM recap): boxes B^l_alpha of an octree with
centres c^l_alpha and size a_l, levels l = 0 (root) .. L, highest active level 2
(Table "Notation"); the interaction list I(B^l_alpha) = boxes of level l that are
not neighbours of B^l_alpha but whose parent is a neighbour of the parent of
B^l_alpha (M2L paragraph); the neighbour list N(B^L_alpha) = B^L_alpha and all
its neighbours (after Eq. FMM_FinalStep).

The paper uses uniform trees and leaves these conventions open; the ones taken
here are fixed so that an independent implementation can reproduce the tree bit
for bit:

* root cube: given explicitly, or centred on the bounding box of all points
  with side = the largest extent (1 if that is 0);
* box index at depth D: clamp(floor((x - corner) * (2^D / side)), 0, 2^D - 1);
  coarser levels take the index shifted right;
* box centre c = corner + (idx + 1/2) * (side / 2^l), box size a_l = side / 2^l;
* only boxes holding at least one source or target exist (sparse, level uniform);
* adaptive trees (max_leaf given): a box of level l < depth is split into its
  children only when l < 2 (the far field starts at level 2), when it holds more than
  max_leaf sources or more than max_leaf targets, or when it is crowded: it holds a
  point and the other cubes of level l within Chebyshev distance b of it (occupied or
  not by boxes of the tree) hold more than (2b+1)^3 max_leaf sources or more than that
  many targets -- a leaf of level l < depth then sums at most
  ((2b+1)^3 + 1 + l ((2b+1)^3 - 1)) max_leaf sources directly (its own, the other cubes
  around it, and at most (2b+1)^3 - 1 leaves per coarser level).  The other boxes are leaves, so
  leaves lie on several levels and no box exists below a leaf.  A target leaf B
  and a source leaf C interact directly (P2P) when their ancestors at the coarser
  of their two levels, m = min(l_B, l_C), are neighbours; otherwise the ancestors
  first stop being neighbours at some level l0 <= m, where the source ancestor is in
  the interaction list of the target ancestor (M2L).  This takes the U list and the
  W and X lists of adaptive FMMs as direct interactions and keeps M2L between boxes
  of one level, so the diagonal transfer of Section 3 is used unchanged (the paper
  treats uniform trees only);
* boxes and points are ordered by Morton key (x bit above y bit above z bit),
  points by key and then by original index;
* "neighbour" = Chebyshev distance of box indices <= b, b the number of buffer
  boxes (Section 3.3.3: b = 1, the common case, or 2, so that |r0| >= (b + 1) a_l);
  a box is its own neighbour.  The interaction list of a box then holds the
  children of its parent's neighbours that are not its own neighbours, at offsets
  (di, dj, dk) = idx(source box) - idx(target box) in [-D, D]^3, D = 2b + 1;
  transfer-vector index v = (di+D) W^2 + (dj+D) W + (dk+D), W = 2D + 1 (b = 1:
  v = (di+3)*49 + (dj+3)*7 + (dk+3), 316 vectors; b = 2: W = 11, 1206 vectors).

Everything is plain Python / numpy on float64 and int64.
"""
import numpy as np

MAX_DEPTH = 20


def root_cube(points, root=None):
    """Return (corner[3], side) of the root box."""
    if root is not None:
        return np.array(root[:3], dtype=np.float64), float(root[3])
    lo = points.min(axis=0)
    hi = points.max(axis=0)
    side = float(np.max(hi - lo))
    if side == 0.0:
        side = 1.0
    corner = (lo + hi) / 2.0 - side / 2.0
    return corner, side


def box_index(points, corner, side, depth):
    """Integer box coordinates (n, 3) of each point at the given depth."""
    nb = 2 ** depth
    scale = float(nb) / side
    v = np.floor((points - corner) * scale)
    v = np.clip(v, 0.0, float(nb - 1))
    return v.astype(np.int64)


def morton_key(idx, depth):
    """Interleave the bits of (ix, iy, iz); x is the most significant of each triple."""
    key = np.zeros(idx.shape[0], dtype=np.int64)
    for b in range(depth):
        key |= ((idx[:, 0] >> b) & 1) << (3 * b + 2)
        key |= ((idx[:, 1] >> b) & 1) << (3 * b + 1)
        key |= ((idx[:, 2] >> b) & 1) << (3 * b)
    return key


def max_occupancy(sources, targets, corner, side, depth):
    occ = 0
    for pts in (sources, targets):
        if pts.shape[0] == 0:
            continue
        key = morton_key(box_index(pts, corner, side, depth), depth)
        _, counts = np.unique(key, return_counts=True)
        occ = max(occ, int(counts.max()))
    return occ


def occupancy_depth(sources, targets, corner, side, max_leaf):
    """Smallest depth D whose fullest box holds <= max_leaf sources and <= max_leaf targets."""
    for d in range(MAX_DEPTH + 1):
        if max_occupancy(sources, targets, corner, side, d) <= max_leaf:
            return d
    return MAX_DEPTH


def transfer_span(buffer=1):
    """(D, W): offsets lie in [-D, D]^3, D = 2 buffer + 1; W = 2 D + 1 index values per axis."""
    D = 2 * buffer + 1
    return D, 2 * D + 1


def transfer_index(d, buffer=1):
    """Index 0..W^3-1 of a box offset (di, dj, dk), each in [-D, D] (b = 1: 0..342)."""
    D, W = transfer_span(buffer)
    return (d[0] + D) * W * W + (d[1] + D) * W + (d[2] + D)


def transfer_offset(v, buffer=1):
    """Inverse of transfer_index."""
    D, W = transfer_span(buffer)
    return np.array([v // (W * W) - D, (v // W) % W - D, v % W - D], dtype=np.int64)


class Tree:
    """Sparse octree over sources and targets, levels 0..depth: level uniform, or adaptive
    (leaves on several levels) when max_leaf is given.

    Attributes
    ----------
    corner, side, depth
    src_perm, tgt_perm : original indices of sources / targets in tree order
    levels[l] : dict with 'idx' (n,3) int64, 'key' (n,), 'center' (n,3),
                'parent' (n,) position of the parent box in levels[l-1]
    src_start/src_count, tgt_start/tgt_count : point ranges of the depth-level
                boxes inside the permuted point arrays
    ilist[l], vlist[l] : for l >= 2, per box, the interaction-list box positions
                (ascending) and their transfer-vector indices
    nlist : per leaf, the leaves it interacts with directly (ascending)
    buffer : number of buffer boxes (1 or 2)
    leaf_level, leaf_box : level and position in that level of every leaf, in Morton
                order of their points (a uniform tree's leaves are the depth-level boxes)
    levels[l] also holds per box 'src_start', 'src_count', 'tgt_start', 'tgt_count'
                (the points of its whole subtree, contiguous in tree order), 'split'
                (has children) and 'leaf'
    """

    def __init__(self, sources, targets, depth, root=None, buffer=1, max_leaf=None):
        self.buffer = int(buffer)
        self.max_leaf = None if max_leaf is None else int(max_leaf)
        adaptive = self.max_leaf is not None
        sources = np.asarray(sources, dtype=np.float64).reshape(-1, 3)
        targets = np.asarray(targets, dtype=np.float64).reshape(-1, 3)
        allp = np.concatenate([sources, targets], axis=0)
        self.corner, self.side = root_cube(allp, root)
        self.depth = int(depth)
        D = self.depth
        sidx = box_index(sources, self.corner, self.side, D)
        tidx = box_index(targets, self.corner, self.side, D)
        skey = morton_key(sidx, D)
        tkey = morton_key(tidx, D)
        # stable sort by key, ties by original index
        self.src_perm = np.lexsort((np.arange(len(skey)), skey))
        self.tgt_perm = np.lexsort((np.arange(len(tkey)), tkey))
        skey_sorted = skey[self.src_perm]
        tkey_sorted = tkey[self.tgt_perm]

        # boxes per level
        leaf_keys = np.unique(np.concatenate([skey, tkey]))
        self.levels = []
        for l in range(D + 1):
            keys_l = np.unique(leaf_keys >> (3 * (D - l)))
            if adaptive and l > 0:
                # boxes exist only below split boxes
                up = self.levels[l - 1]
                pos = np.minimum(np.searchsorted(up['key'], keys_l >> 3), len(up['key']) - 1)
                keys_l = keys_l[(up['key'][pos] == (keys_l >> 3)) & up['split'][pos]]
            idx = np.zeros((len(keys_l), 3), dtype=np.int64)
            for b in range(l):
                idx[:, 0] |= ((keys_l >> (3 * b + 2)) & 1) << b
                idx[:, 1] |= ((keys_l >> (3 * b + 1)) & 1) << b
                idx[:, 2] |= ((keys_l >> (3 * b)) & 1) << b
            h = self.side / float(2 ** l)
            center = self.corner + (idx.astype(np.float64) + 0.5) * h
            if l == 0:
                parent = np.full(len(keys_l), -1, dtype=np.int64)
            else:
                pkeys = self.levels[l - 1]['key']
                parent = np.searchsorted(pkeys, keys_l >> 3).astype(np.int64)
            sh = 3 * (D - l)
            s0 = np.searchsorted(skey_sorted >> sh, keys_l, side='left')
            sc = np.searchsorted(skey_sorted >> sh, keys_l, side='right') - s0
            t0 = np.searchsorted(tkey_sorted >> sh, keys_l, side='left')
            tc = np.searchsorted(tkey_sorted >> sh, keys_l, side='right') - t0
            if adaptive:
                crowd = self._crowded(idx, sc + tc, skey_sorted >> sh, tkey_sorted >> sh, l)
                split = (l < D) & ((l < 2) | (sc > self.max_leaf) | (tc > self.max_leaf) | crowd)
            else:
                split = np.full(len(keys_l), l < D)
            self.levels.append({'idx': idx, 'key': keys_l, 'center': center,
                                'parent': parent, 'a': h,
                                'src_start': s0, 'src_count': sc, 'tgt_start': t0, 'tgt_count': tc,
                                'split': split, 'leaf': ~split})

        # leaves of all levels in Morton order of their first depth-level key
        lv = np.concatenate([np.full(int(L['leaf'].sum()), l, dtype=np.int64)
                             for l, L in enumerate(self.levels)])
        bx = np.concatenate([np.nonzero(L['leaf'])[0] for L in self.levels]).astype(np.int64)
        first = np.array([int(self.levels[l]['key'][b]) << (3 * (D - l)) for l, b in zip(lv, bx)],
                         dtype=np.int64)
        order = np.argsort(first, kind='stable')
        self.leaf_level, self.leaf_box = lv[order], bx[order]
        pick = lambda f: np.array([self.levels[l][f][b] for l, b in zip(self.leaf_level, self.leaf_box)],
                                  dtype=np.int64)
        self.src_start, self.src_count = pick('src_start'), pick('src_count')
        self.tgt_start, self.tgt_count = pick('tgt_start'), pick('tgt_count')
        self._leaf_idx = np.array([self.levels[l]['idx'][b] for l, b in zip(self.leaf_level, self.leaf_box)],
                                  dtype=np.int64).reshape(-1, 3)

        # lists, built per box on first use (ilist[l][a], vlist[l][a], nlist[a])
        self._where = {}
        self._ilists = {}
        self.ilist = [None] * (D + 1)
        self.vlist = [None] * (D + 1)
        for l in range(2, D + 1):
            n = len(self.levels[l]['key'])
            self.ilist[l] = _PerBox(n, lambda a, l=l: self._interaction_list(l, a)[0])
            self.vlist[l] = _PerBox(n, lambda a, l=l: self._interaction_list(l, a)[1])
        if adaptive:
            self.nlist = _PerBox(len(self.leaf_level), self._adaptive_neighbours)
        else:
            self.nlist = _PerBox(len(self.levels[D]['key']), lambda a: self._neighbour_list(D, a))

    def _crowded(self, idx, count, skeys, tkeys, l):
        """Per box: holds a point and the other level-l cubes within Chebyshev distance b hold
        more than (2b+1)^3 max_leaf sources or targets (skeys, tkeys: sorted level-l keys of
        all sources and targets)."""
        bw, nb = self.buffer, 2 ** l
        lim = (2 * bw + 1) ** 3 * self.max_leaf

        def points_in(keys, sorted_keys):
            return np.searchsorted(sorted_keys, keys, side='right') - np.searchsorted(sorted_keys, keys, side='left')

        cs = np.zeros(len(idx), dtype=np.int64)
        ct = np.zeros(len(idx), dtype=np.int64)
        for d in np.ndindex(2 * bw + 1, 2 * bw + 1, 2 * bw + 1):
            off = np.array(d) - bw
            if not off.any():
                continue
            c = idx + off
            inside = np.all((c >= 0) & (c < nb), axis=1)
            k = morton_key(np.clip(c, 0, nb - 1), l)
            cs += np.where(inside, points_in(k, skeys), 0)
            ct += np.where(inside, points_in(k, tkeys), 0)
        return (count > 0) & ((cs > lim) | (ct > lim))

    def _adaptive_neighbours(self, g):
        """Leaves C whose ancestor at level min(l_B, l_C) neighbours leaf g's ancestor there."""
        lb, lc = int(self.leaf_level[g]), self.leaf_level
        m = np.minimum(lb, lc)
        ab = self._leaf_idx[g][None, :] >> (lb - m)[:, None]
        ac = self._leaf_idx >> (lc - m)[:, None]
        return np.nonzero(np.max(np.abs(ab - ac), axis=1) <= self.buffer)[0].astype(np.int64)

    def _lookup(self, l):
        if l not in self._where:
            self._where[l] = {tuple(int(c) for c in self.levels[l]['idx'][i]): i
                              for i in range(len(self.levels[l]['key']))}
        return self._where[l]

    def _interaction_list(self, l, a):
        """(box positions, transfer-vector indices) of I(box a at level l), by Morton key."""
        if (l, a) in self._ilists:
            return self._ilists[(l, a)]
        lev = self.levels[l]
        where = self._lookup(l)
        nb = 2 ** l
        bw = self.buffer
        span = 2 * bw + 1
        ia = lev['idx'][a]
        pa = ia >> 1
        found = []
        # children of the parent's neighbours (Chebyshev distance <= buffer)
        for dp in np.ndindex(span, span, span):
            pn = pa + np.array(dp) - bw
            for dc in np.ndindex(2, 2, 2):
                ib = pn * 2 + np.array(dc)
                if np.any(ib < 0) or np.any(ib >= nb):
                    continue
                d = ib - ia
                if np.max(np.abs(d)) <= bw:
                    continue
                b = where.get(tuple(int(c) for c in ib))
                if b is not None:
                    found.append((lev['key'][b], b, transfer_index(d, bw)))
        found.sort()
        out = (np.array([f[1] for f in found], dtype=np.int64),
               np.array([f[2] for f in found], dtype=np.int64))
        self._ilists[(l, a)] = out
        return out

    def _neighbour_list(self, l, a):
        lev = self.levels[l]
        where = self._lookup(l)
        bw = self.buffer
        span = 2 * bw + 1
        ia = lev['idx'][a]
        found = []
        for d in np.ndindex(span, span, span):
            ib = ia + np.array(d) - bw
            b = where.get(tuple(int(c) for c in ib))
            if b is not None:
                found.append((lev['key'][b], b))
        found.sort()
        return np.array([f[1] for f in found], dtype=np.int64)


class _PerBox:
    """Per-box lists computed by `fn(box)` on first access and kept (indexable, iterable)."""

    def __init__(self, n, fn):
        self.n, self.fn, self.cache = n, fn, {}

    def __len__(self):
        return self.n

    def __getitem__(self, a):
        a = int(a)
        if a < 0:
            a += self.n
        if not 0 <= a < self.n:
            raise IndexError(a)
        if a not in self.cache:
            self.cache[a] = self.fn(a)
        return self.cache[a]

    def __iter__(self):
        return (self[a] for a in range(self.n))
