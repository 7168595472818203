"""Cluster tree (Algorithm 1) and block tree (Algorithm 2) of an H-matrix.

Cluster tree (Sec. 2, Algorithm 1): the bounding box of a cluster is the box of
the supports (triangle vertices) of its degrees of freedom.  A cluster with more
than C_lf degrees of freedom is split along the longest side of its box (ties:
lowest axis) at the side's midpoint; a degree of freedom goes to the first son
when its centroid coordinate is below the midpoint.  If one side would be
empty the split falls back to the median (ties broken by original index).
Degrees of freedom are stored first son first, which defines the permutation
`perm` (cluster order -> original index).  Clusters are numbered in pre-order,
so every cluster's index range [begin, begin+size) is contiguous.

Block tree (Sec. 2, Algorithm 2): a block (t, s) is admissible when
min(diam t, diam s) <= eta * dist(t, s) with dist > 0 (the paper prints the
eta = 1 form), where diam is the box diagonal and dist the Euclidean distance
of the boxes.  An admissible block is a low-rank leaf; otherwise the block is
split into sons(t) x sons(s) when both clusters have sons, else it is a dense
leaf.
"""
from __future__ import annotations

import numpy as np


class ClusterTree:
    """Flat pre-order cluster arrays.

    begin, size, son0, son1 (-1 for a leaf), level, bmin/bmax (n_clusters,3),
    perm (n,) cluster position -> original DoF.
    """

    def __init__(self, begin, size, son0, son1, level, bmin, bmax, perm):
        self.begin = np.asarray(begin, dtype=np.int32)
        self.size = np.asarray(size, dtype=np.int32)
        self.son0 = np.asarray(son0, dtype=np.int32)
        self.son1 = np.asarray(son1, dtype=np.int32)
        self.level = np.asarray(level, dtype=np.int32)
        self.bmin = np.asarray(bmin, dtype=np.float64)
        self.bmax = np.asarray(bmax, dtype=np.float64)
        self.perm = np.asarray(perm, dtype=np.int32)

    @property
    def n(self):
        return int(self.perm.shape[0])

    @property
    def n_clusters(self):
        return int(self.begin.shape[0])

    def is_leaf(self, t):
        return self.son0[t] < 0

    def diam(self, t):
        return float(np.linalg.norm(self.bmax[t] - self.bmin[t]))

    def dist(self, t, s):
        gap = np.maximum(0.0, np.maximum(self.bmin[s] - self.bmax[t], self.bmin[t] - self.bmax[s]))
        return float(np.linalg.norm(gap))


def build_cluster_tree(centroid, lo, hi, leaf_size):
    """Algorithm 1 (setup_clustertree) on triangle centroids and supports."""
    n = centroid.shape[0]
    begin, size, son0, son1, level, bmin, bmax = [], [], [], [], [], [], []
    perm = np.empty(n, dtype=np.int64)

    # explicit stack of (dof array, begin position, level, parent slot)
    def new_cluster(dofs, pos, lev):
        idx = len(begin)
        begin.append(pos)
        size.append(len(dofs))
        son0.append(-1)
        son1.append(-1)
        level.append(lev)
        bmin.append(lo[dofs].min(axis=0))
        bmax.append(hi[dofs].max(axis=0))
        return idx

    def setup(dofs, pos, lev):
        t = new_cluster(dofs, pos, lev)
        if len(dofs) > leaf_size:
            ext = bmax[t] - bmin[t]
            d = int(np.argmax(ext))  # argmax returns the lowest axis on ties
            midv = 0.5 * (bmin[t][d] + bmax[t][d])
            c = centroid[dofs, d]
            first = dofs[c < midv]
            second = dofs[c >= midv]
            if len(first) == 0 or len(second) == 0:
                order = np.lexsort((dofs, c))  # by coordinate, then original index
                srt = dofs[order]
                h = len(dofs) // 2
                first, second = srt[:h], srt[h:]
            s0 = setup(first, pos, lev + 1)
            s1 = setup(second, pos + len(first), lev + 1)
            son0[t] = s0
            son1[t] = s1
        else:
            perm[pos:pos + len(dofs)] = dofs
        return t

    import sys
    old = sys.getrecursionlimit()
    sys.setrecursionlimit(max(old, 10000))
    try:
        setup(np.arange(n, dtype=np.int64), 0, 0)
    finally:
        sys.setrecursionlimit(old)
    return ClusterTree(begin, size, son0, son1, level, np.array(bmin), np.array(bmax), perm)


class BlockLeaves:
    """Leaves of the block tree, in the depth-first order of Algorithm 2
    (sons visited (t0,s0), (t0,s1), (t1,s0), (t1,s1)).  kind: 0 dense, 1 low-rank."""

    def __init__(self, row_cl, col_cl, kind):
        self.row_cl = np.asarray(row_cl, dtype=np.int32)
        self.col_cl = np.asarray(col_cl, dtype=np.int32)
        self.kind = np.asarray(kind, dtype=np.int8)

    def __len__(self):
        return int(self.row_cl.shape[0])


def admissible(ct, t, s, eta):
    d = ct.dist(t, s)
    return d > 0.0 and min(ct.diam(t), ct.diam(s)) <= eta * d


def build_block_leaves(ct, eta):
    """Algorithm 2 (setup_blocktree) from (root, root); returns the leaf list."""
    rows, cols, kinds = [], [], []
    stack = [(0, 0)]
    while stack:
        t, s = stack.pop()
        if admissible(ct, t, s, eta):
            rows.append(t); cols.append(s); kinds.append(1)
        elif ct.son0[t] >= 0 and ct.son0[s] >= 0:
            # pushed in reverse so that (t0,s0) is processed first
            stack.append((ct.son1[t], ct.son1[s]))
            stack.append((ct.son1[t], ct.son0[s]))
            stack.append((ct.son0[t], ct.son1[s]))
            stack.append((ct.son0[t], ct.son0[s]))
        else:
            rows.append(t); cols.append(s); kinds.append(0)
    return BlockLeaves(rows, cols, kinds)
