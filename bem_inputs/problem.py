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
from .mesh import ellipsoid, icosphere, triangle_data
from .trees import ClusterTree, build_block_leaves, build_cluster_tree

CACHE_VERSION = 3


class Problem:
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


def _cache_dir():
    d = os.environ.get("HLU_CACHE_DIR") or os.path.join(os.path.expanduser("~"), ".cache", "hlu_gb300")
    os.makedirs(d, exist_ok=True)
    return d


def _key(**kw):
    s = repr(sorted(kw.items())) + f"v{CACHE_VERSION}"
    return hashlib.sha1(s.encode()).hexdigest()[:16]


def build_problem(r, leaf, eta, eps, nrhs=1, seed=0, axes=None, cache=True, verbose=False):
    """Build (or load from the on-disk cache) the seeded BEM H-matrix problem.

    r     refinement steps of the icosahedron (n = 20 * 4**r)
    leaf  C_lf, the cluster-tree leaf size
    eta   admissibility parameter
    eps   ACA / recompression tolerance
    nrhs  number of right-hand sides, b = default_rng(seed).standard_normal((nrhs, n)).T
    axes  None for the unit sphere, else ellipsoid axes (ax, ay, az)
    """
    key = _key(r=r, leaf=leaf, eta=float(eta), eps=float(eps), nrhs=nrhs, seed=seed,
               axes=None if axes is None else tuple(float(a) for a in axes))
    path = os.path.join(_cache_dir(), f"hmat_{key}.npz") if cache else None
    if path and os.path.exists(path):
        try:
            return _load(path)
        except Exception:
            pass
    t0 = time.time()
    v, f = icosphere(r) if axes is None else ellipsoid(r, axes)
    centroid, area, lo, hi = triangle_data(v, f)
    n = centroid.shape[0]
    tree = build_cluster_tree(centroid, lo, hi, leaf)
    bl = build_block_leaves(tree, eta)
    perm = tree.perm.astype(np.int64)

    rank = np.zeros(len(bl), dtype=np.int32)
    kind = bl.kind.copy()
    chunks = []
    fallbacks = 0
    rng_check = np.random.default_rng(12345)
    for l in range(len(bl)):
        t, s = int(bl.row_cl[l]), int(bl.col_cl[l])
        rows = perm[tree.begin[t]:tree.begin[t] + tree.size[t]]
        cols = perm[tree.begin[s]:tree.begin[s] + tree.size[s]]
        if kind[l] == 1:
            U, V = aca_partial(centroid, area, rows, cols, eps)
            ok = U.shape[1] <= min(len(rows), len(cols)) // 2
            if ok:
                U, V = recompress(U, V, eps)
                ii = rng_check.integers(0, len(rows), 64)
                jj = rng_check.integers(0, len(cols), 64)
                exact = kernel_block(centroid, area, rows[ii], cols[jj])[np.arange(64), np.arange(64)]
                approx = np.einsum("ik,ik->i", U[ii], V[jj])
                ok = np.max(np.abs(exact - approx)) <= 10.0 * eps * np.max(np.abs(exact))
                if not ok:
                    fallbacks += 1
            if ok:
                rank[l] = U.shape[1]
                chunks.append(np.asfortranarray(U).ravel(order="F"))
                chunks.append(np.asfortranarray(V).ravel(order="F"))
                continue
            kind[l] = 0
        chunks.append(kernel_block(centroid, area, rows, cols).ravel(order="F"))
    sizes = np.array([c.shape[0] for c in chunks], dtype=np.int64)
    # one leaf may own two chunks (U and V): rebuild offsets per leaf
    offset = np.zeros(len(bl), dtype=np.int64)
    pos = 0
    ci = 0
    for l in range(len(bl)):
        offset[l] = pos
        if kind[l] == 1:
            pos += sizes[ci] + sizes[ci + 1]
            ci += 2
        else:
            pos += sizes[ci]
            ci += 1
    data = np.concatenate(chunks) if chunks else np.zeros(0)
    rng = np.random.default_rng(seed)
    b = np.asfortranarray(rng.standard_normal((nrhs, n)).T)
    p = Problem(n=n, r=r, leaf=leaf, eta=float(eta), eps=float(eps), nrhs=nrhs, seed=seed,
                axes=axes, tree=tree, row_cl=bl.row_cl, col_cl=bl.col_cl, kind=kind,
                rank=rank, offset=offset, data=data, b=b, centroid=centroid, area=area,
                aca_fallbacks=fallbacks, build_seconds=time.time() - t0)
    if verbose:
        print(f"built n={n} leaves={len(bl)} in {p.build_seconds:.1f}s")
    if path:
        _save(path, p)
    return p


_ARRAYS = ("row_cl", "col_cl", "kind", "rank", "offset", "data", "b", "centroid", "area")
_TREE = ("begin", "size", "son0", "son1", "level", "bmin", "bmax", "perm")
_SCAL = ("n", "r", "leaf", "eta", "eps", "nrhs", "seed", "aca_fallbacks", "build_seconds")


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
        kw[k] = z["s_" + k].item()
    ax = z["s_axes"]
    kw["axes"] = None if ax.size == 0 else tuple(ax.tolist())
    return Problem(tree=tree, **kw)
