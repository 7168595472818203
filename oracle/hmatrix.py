"""The oracle's own H-matrix representation (test infrastructure only).

An HBlock mirrors the paper's `hmatrix` record (Sec. 2): a block (t, s) of the
row cluster t and column cluster s that is either dense (`amatrix`), low rank
(`rkmatrix`, X = U V^T with k columns, Sec. 3.1) or partitioned into
sons(t) x sons(s).  It is rebuilt here from the shared leaf arrays: the block
tree is the one of Algorithm 2, recovered top-down from (root, root) - a block
is a leaf exactly when it appears in the leaf list, otherwise both clusters
have two sons and the block has four sons.
"""
from __future__ import annotations

import numpy as np


class HBlock:
    __slots__ = ("t", "s", "r0", "m", "c0", "n", "kind", "D", "U", "V", "sons", "leaf_id")

    def __init__(self, t, s, r0, m, c0, n):
        self.t, self.s = t, s
        self.r0, self.m, self.c0, self.n = r0, m, c0, n
        self.kind = None  # "dense" | "lowrank" | "part"
        self.D = self.U = self.V = None
        self.sons = None  # [[b00, b01], [b10, b11]]
        self.leaf_id = -1

    @property
    def rank(self):
        return self.U.shape[1] if self.kind == "lowrank" else None

    def leaves(self):
        if self.kind == "part":
            for row in self.sons:
                for b in row:
                    yield from b.leaves()
        else:
            yield self


def build_hmatrix(problem, copy=True):
    """Block tree of the problem with the leaf data copied into FP64 arrays."""
    tree = problem.tree
    index = {}
    for l in range(problem.n_leaves):
        index[(int(problem.row_cl[l]), int(problem.col_cl[l]))] = l

    def make(t, s):
        b = HBlock(t, s, int(tree.begin[t]), int(tree.size[t]), int(tree.begin[s]), int(tree.size[s]))
        l = index.get((t, s))
        if l is not None:
            b.leaf_id = l
            if problem.kind[l] == 0:
                b.kind = "dense"
                b.D = np.array(problem.leaf_dense(l), dtype=np.float64, order="C", copy=True)
            else:
                b.kind = "lowrank"
                U, V = problem.leaf_factors(l)
                b.U = np.array(U, dtype=np.float64, copy=True)
                b.V = np.array(V, dtype=np.float64, copy=True)
            return b
        t0, t1 = int(tree.son0[t]), int(tree.son1[t])
        s0, s1 = int(tree.son0[s]), int(tree.son1[s])
        if t0 < 0 or s0 < 0:
            raise ValueError(f"block ({t},{s}) is neither a leaf nor splittable")
        b.kind = "part"
        b.sons = [[make(t0, s0), make(t0, s1)], [make(t1, s0), make(t1, s1)]]
        return b

    return make(0, 0)


def densify(b):
    """Dense m x n array of a block (Sec. 3.1: X = U V^T for low-rank)."""
    if b.kind == "dense":
        return b.D.copy()
    if b.kind == "lowrank":
        return b.U @ b.V.T
    out = np.empty((b.m, b.n))
    for row in b.sons:
        for c in row:
            out[c.r0 - b.r0:c.r0 - b.r0 + c.m, c.c0 - b.c0:c.c0 - b.c0 + c.n] = densify(c)
    return out


def hmul(b, x):
    """b @ x for a dense block x with b.n rows (exact; Sec. 3.1 low-rank matvec
    y = U (V^T x) on low-rank leaves)."""
    if b.kind == "dense":
        return b.D @ x
    if b.kind == "lowrank":
        return b.U @ (b.V.T @ x)
    out = np.zeros((b.m,) + x.shape[1:])
    for row in b.sons:
        for c in row:
            out[c.r0 - b.r0:c.r0 - b.r0 + c.m] += hmul(c, x[c.c0 - b.c0:c.c0 - b.c0 + c.n])
    return out


def hmul_t(b, x):
    """b^T @ x for a dense block x with b.m rows (exact)."""
    if b.kind == "dense":
        return b.D.T @ x
    if b.kind == "lowrank":
        return b.V @ (b.U.T @ x)
    out = np.zeros((b.n,) + x.shape[1:])
    for row in b.sons:
        for c in row:
            out[c.c0 - b.c0:c.c0 - b.c0 + c.n] += hmul_t(c, x[c.r0 - b.r0:c.r0 - b.r0 + c.m])
    return out
