"""Seeded synthetic H-matrix problems (the inputs every solver consumes).

A Problem bundles the cluster tree, the block-tree leaves with their data in
the flat layout below, the right-hand sides and the geometry.  Building it uses
mesh refinement, Algorithms 1 and 2, ACA and SVD recompression; none of the
H-LU arithmetic (factorisation, triangular solves, truncated products) is here.

Leaf layout (shared, data only):
    row_cl[l], col_cl[l]  cluster ids (pre-order numbering of the cluster tree)
    kind[l]               0 dense, 1 low-rank
    rank[l]               k for low-rank leaves, 0 for dense
    offset[l]             first double of the leaf in `data`
    data                  dense: m x n column-major; low-rank: U (m x k) then V (n x k)
Matrix rows and columns are numbered in cluster order: position p holds the
original degree of freedom perm[p].
"""
from __future__ import annotations

import hashlib
import os
import time

import numpy as np

from .assemble import aca_partial, kernel_block, recompress
from .mesh import ellipse_panels, ellipsoid, icosphere, interval_cells, triangle_data
from .trees import BlockLeaves, ClusterTree, admissible, build_block_leaves, build_cluster_tree

CACHE_VERSION = 4


class Problem:
    dim = 3  # problems cached before the d = 1, 2 kernels existed are d = 3
    def __init__(self, **kw):
        self.__dict__.update(kw)

    # ------------------------------------------------------------------ sizes
    @property
    def n_leaves(self):
        return int(self.row_cl.shape[0])

    def leaf_shape(self, l):
        t, s = int(self.row_cl[l]), int(self.col_cl[l])
        return int(self.tree.size[t]), int(self.tree.size[s])

    def leaf_ranges(self, l):
        t, s = int(self.row_cl[l]), int(self.col_cl[l])
        return (int(self.tree.begin[t]), int(self.tree.size[t]),
                int(self.tree.begin[s]), int(self.tree.size[s]))

    def leaf_dense(self, l):
        """The stored dense leaf (m x n view) - kind 0 only."""
        m, n = self.leaf_shape(l)
        o = int(self.offset[l])
        return self.data[o:o + m * n].reshape((m, n), order="F")

    def leaf_factors(self, l):
        """(U m x k, V n x k) views of a stored low-rank leaf - kind 1 only."""
        m, n = self.leaf_shape(l)
        k = int(self.rank[l])
        o = int(self.offset[l])
        U = self.data[o:o + m * k].reshape((m, k), order="F")
        V = self.data[o + m * k:o + (m + n) * k].reshape((n, k), order="F")
        return U, V

    def storage_doubles(self):
        return int(self.data.shape[0])

    def rank_histogram(self):
        lr = self.kind == 1
        return np.bincount(self.rank[lr]) if lr.any() else np.zeros(1, dtype=np.int64)

    def b_perm(self):
        """Right-hand sides in cluster order."""
        return self.b[self.tree.perm]


def sub_problem(p, cluster):
    """The diagonal block (cluster, cluster) of p as a problem of its own: the
    sub-tree of `cluster` renumbered in pre-order, the leaves inside the block
    with their data copied, b restricted to the block's rows.  (A data-layout
    operation: the leaves are the same matrix blocks.)"""
    t = p.tree
    order = []
    stack = [int(cluster)]
    while stack:
        c = stack.pop()
        order.append(c)
        if t.son0[c] >= 0:
            stack.append(int(t.son1[c]))
            stack.append(int(t.son0[c]))
    new_id = {c: i for i, c in enumerate(order)}
    b0, m = int(t.begin[cluster]), int(t.size[cluster])
    orig = t.perm[b0:b0 + m].astype(np.int64)
    rank_of = np.empty(m, dtype=np.int64)
    rank_of[np.argsort(orig, kind="stable")] = np.arange(m)
    tree = ClusterTree(
        begin=[int(t.begin[c]) - b0 for c in order], size=[int(t.size[c]) for c in order],
        son0=[new_id[int(t.son0[c])] if t.son0[c] >= 0 else -1 for c in order],
        son1=[new_id[int(t.son1[c])] if t.son1[c] >= 0 else -1 for c in order],
        level=[int(t.level[c]) - int(t.level[cluster]) for c in order],
        bmin=t.bmin[order], bmax=t.bmax[order], perm=rank_of)
    keep = [l for l in range(p.n_leaves) if int(p.row_cl[l]) in new_id and int(p.col_cl[l]) in new_id]
    chunks, offset = [], []
    pos = 0
    for l in keep:
        mm, nn = p.leaf_shape(l)
        size = mm * nn if p.kind[l] == 0 else (mm + nn) * int(p.rank[l])
        o = int(p.offset[l])
        chunks.append(p.data[o:o + size])
        offset.append(pos)
        pos += size
    return Problem(n=m, r=p.r, leaf=p.leaf, eta=p.eta, eps=p.eps, nrhs=p.nrhs, seed=p.seed, axes=p.axes,
                   tree=tree, row_cl=np.array([new_id[int(p.row_cl[l])] for l in keep], dtype=np.int32),
                   col_cl=np.array([new_id[int(p.col_cl[l])] for l in keep], dtype=np.int32),
                   kind=p.kind[keep].copy(), rank=p.rank[keep].copy(), offset=np.array(offset, dtype=np.int64),
                   data=np.concatenate(chunks), b=np.asfortranarray(p.b[orig]),
                   centroid=p.centroid[orig], area=p.area[orig], aca_fallbacks=0, build_seconds=0.0)


def _cache_dir():
    d = os.environ.get("HLU_CACHE_DIR") or os.path.join(os.path.expanduser("~"), ".cache", "hlu_gb300")
    os.makedirs(d, exist_ok=True)
    return d


def _key(**kw):
    s = repr(sorted(kw.items())) + f"v{CACHE_VERSION}"
    return hashlib.sha1(s.encode()).hexdigest()[:16]


def build_problem(r, leaf, eta, eps, nrhs=1, seed=0, axes=None, cache=True, verbose=False, dim=3):
    """Build (or load from the on-disk cache) the seeded BEM H-matrix problem.

    r     size: n = 20 * 4**r (refinement steps of the icosahedron for dim = 3)
    leaf  C_lf, the cluster-tree leaf size
    eta   admissibility parameter (0: no admissible block, every leaf dense)
    eps   ACA / recompression tolerance
    nrhs  number of right-hand sides, b = default_rng(seed).standard_normal((nrhs, n)).T
    axes  dim 3: None for the unit sphere, else ellipsoid axes (ax, ay, az);
          dim 2: the ellipse's semi-axes (default (0.5, 0.5)); dim 1: unused
    dim   3: surface of a sphere or ellipsoid, kernel 1 / (4 pi |x - y|);
          2: closed curve, kernel -log|x - y| / (2 pi); 1: interval [0, 1], kernel -log|x - y|
    """
    kw = dict(r=r, leaf=leaf, eta=float(eta), eps=float(eps), nrhs=nrhs, seed=seed,
              axes=None if axes is None else tuple(float(a) for a in axes))
    if dim != 3:
        kw["dim"] = int(dim)
    key = _key(**kw)
    path = os.path.join(_cache_dir(), f"hmat_{key}.npz") if cache else None
    if path and os.path.exists(path):
        try:
            return _load(path)
        except Exception:
            pass
    t0 = time.time()
    if dim == 3:
        v, f = icosphere(r) if axes is None else ellipsoid(r, axes)
        centroid, area, lo, hi = triangle_data(v, f)
    elif dim == 2:
        centroid, area, lo, hi = ellipse_panels(20 * 4 ** r, (0.5, 0.5) if axes is None else axes)
    elif dim == 1:
        centroid, area, lo, hi = interval_cells(20 * 4 ** r)
    else:
        raise ValueError(f"dim must be 1, 2 or 3, got {dim}")
    n = centroid.shape[0]
    tree = build_cluster_tree(centroid, lo, hi, leaf)
    bl = build_block_leaves(tree, eta)
    perm = tree.perm.astype(np.int64)

    rows_out, cols_out, kind_out, rank_out, offset_out, chunks = [], [], [], [], [], []
    pos = 0
    fallbacks = 0
    rng_check = np.random.default_rng(12345)

    def emit(t, s, k, U=None, V=None):
        nonlocal pos
        rows_out.append(t); cols_out.append(s); kind_out.append(k); offset_out.append(pos)
        if k == 1:
            rank_out.append(U.shape[1])
            chunks.append(np.asfortranarray(U).ravel(order="F"))
            chunks.append(np.asfortranarray(V).ravel(order="F"))
            pos += U.size + V.size
        else:
            rank_out.append(0)
            rr = perm[tree.begin[t]:tree.begin[t] + tree.size[t]]
            cc = perm[tree.begin[s]:tree.begin[s] + tree.size[s]]
            chunks.append(kernel_block(centroid, area, rr, cc, dim).ravel(order="F"))
            pos += chunks[-1].size

    def compress(t, s):
        """Low-rank factors of an admissible block, or None when ACA does not
        reach the tolerance with k <= min(m, n) / 2 or fails the sample check."""
        nonlocal fallbacks
        rows = perm[tree.begin[t]:tree.begin[t] + tree.size[t]]
        cols = perm[tree.begin[s]:tree.begin[s] + tree.size[s]]
        U, V = aca_partial(centroid, area, rows, cols, eps, dim)
        if U.shape[1] > min(len(rows), len(cols)) // 2:
            return None
        U, V = recompress(U, V, eps)
        ii = rng_check.integers(0, len(rows), 64)
        jj = rng_check.integers(0, len(cols), 64)
        exact = kernel_block(centroid, area, rows[ii], cols[jj], dim)[np.arange(64), np.arange(64)]
        approx = np.einsum("ik,ik->i", U[ii], V[jj])
        if np.max(np.abs(exact - approx)) > 10.0 * eps * np.max(np.abs(exact)):
            fallbacks += 1
            return None
        return U, V

    def block(t, s, adm):
        # an admissible block is compressed; if compression fails and both
        # clusters have sons it is partitioned like an inadmissible block
        # (Algorithm 2), so a dense leaf always has a leaf cluster on one side
        if adm:
            f = compress(t, s)
            if f is not None:
                emit(t, s, 1, *f)
                return
        if tree.son0[t] >= 0 and tree.son0[s] >= 0:
            for tt in (tree.son0[t], tree.son1[t]):
                for ss in (tree.son0[s], tree.son1[s]):
                    block(int(tt), int(ss), admissible(tree, int(tt), int(ss), eta))
            return
        emit(t, s, 0)

    for l in range(len(bl)):
        block(int(bl.row_cl[l]), int(bl.col_cl[l]), bl.kind[l] == 1)
    kind = np.array(kind_out, dtype=np.int8)
    rank = np.array(rank_out, dtype=np.int32)
    offset = np.array(offset_out, dtype=np.int64)
    bl = BlockLeaves(rows_out, cols_out, kind)
    data = np.concatenate(chunks) if chunks else np.zeros(0)
    rng = np.random.default_rng(seed)
    b = np.asfortranarray(rng.standard_normal((nrhs, n)).T)
    p = Problem(n=n, r=r, leaf=leaf, eta=float(eta), eps=float(eps), nrhs=nrhs, seed=seed,
                axes=axes, dim=int(dim), tree=tree, row_cl=bl.row_cl, col_cl=bl.col_cl, kind=kind,
                rank=rank, offset=offset, data=data, b=b, centroid=centroid, area=area,
                aca_fallbacks=fallbacks, build_seconds=time.time() - t0)
    if verbose:
        print(f"built n={n} leaves={len(bl)} in {p.build_seconds:.1f}s")
    if path:
        _save(path, p)
    return p


def build_structure(r, leaf, eta, eps, nrhs=1, seed=0, axes=None, dim=3):
    """The problem of build_problem without leaf data: geometry, cluster tree (Algorithm 1), the
    block-tree leaves of Algorithm 2 with every admissible block marked low rank (no cross
    approximation is tried, so none falls back to a partitioned or dense block), and the
    right-hand sides.  rank and offset are zero and data is empty: the leaves are to be computed
    elsewhere (the GPU construction, hlu_bem_build)."""
    t0 = time.time()
    if dim == 3:
        v, f = icosphere(r) if axes is None else ellipsoid(r, axes)
        centroid, area, lo, hi = triangle_data(v, f)
    elif dim == 2:
        centroid, area, lo, hi = ellipse_panels(20 * 4 ** r, (0.5, 0.5) if axes is None else axes)
    elif dim == 1:
        centroid, area, lo, hi = interval_cells(20 * 4 ** r)
    else:
        raise ValueError(f"dim must be 1, 2 or 3, got {dim}")
    n = centroid.shape[0]
    tree = build_cluster_tree(centroid, lo, hi, leaf)
    bl = build_block_leaves(tree, eta)
    b = np.asfortranarray(np.random.default_rng(seed).standard_normal((nrhs, n)).T)
    nl = len(bl)
    return Problem(n=n, r=r, leaf=leaf, eta=float(eta), eps=float(eps), nrhs=nrhs, seed=seed,
                   axes=None if axes is None else tuple(float(a) for a in axes), dim=int(dim), tree=tree,
                   row_cl=bl.row_cl, col_cl=bl.col_cl, kind=bl.kind, rank=np.zeros(nl, dtype=np.int32),
                   offset=np.zeros(nl, dtype=np.int64), data=np.zeros(0), b=b, centroid=centroid, area=area,
                   aca_fallbacks=0, build_seconds=time.time() - t0)


_ARRAYS = ("row_cl", "col_cl", "kind", "rank", "offset", "data", "b", "centroid", "area")
_TREE = ("begin", "size", "son0", "son1", "level", "bmin", "bmax", "perm")
_SCAL = ("n", "r", "leaf", "eta", "eps", "nrhs", "seed", "aca_fallbacks", "build_seconds", "dim")


def _save(path, p):
    d = {k: getattr(p, k) for k in _ARRAYS}
    d.update({"tree_" + k: getattr(p.tree, k) for k in _TREE})
    d.update({"s_" + k: np.asarray(getattr(p, k)) for k in _SCAL})
    d["s_axes"] = np.asarray([] if p.axes is None else p.axes, dtype=np.float64)
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, **d)
    os.replace(tmp, path)


def _load(path):
    z = np.load(path)
    tree = ClusterTree(*[z["tree_" + k] for k in _TREE])
    kw = {k: z[k] for k in _ARRAYS}
    kw["b"] = np.asfortranarray(kw["b"])
    for k in _SCAL:
        if "s_" + k in z:
            kw[k] = z["s_" + k].item()
    ax = z["s_axes"]
    kw["axes"] = None if ax.size == 0 else tuple(ax.tolist())
    return Problem(tree=tree, **kw)
