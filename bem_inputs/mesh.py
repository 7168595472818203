"""Surface meshes for the BEM test problems: refined icosahedra (unit sphere) and
ellipsoids.

The paper's experiments discretise boundary integral equations on a surface
(Sec. 6.1); the workloads here use a flat-triangle mesh of the unit sphere.
Construction:

* icosahedron: the 12 vertices are the cyclic permutations of (0, +-1, +-phi),
  scaled to unit length; the 20 faces are the vertex triples that are pairwise
  joined by an edge of the solid (edge length 2 before scaling), oriented so
  that the normal points outwards;
* refinement: each triangle (a, b, c) is cut into four through its edge
  midpoints, the children being ordered (corner a, corner b, corner c,
  centre); every new midpoint is pushed back onto the sphere after each step,
  so r steps give n = 20 * 4**r triangles;
* ellipsoid: the sphere's vertices scaled by the axes (ax, ay, az).

One triangle is one degree of freedom (piecewise-constant collocation).
"""
from __future__ import annotations

import itertools

import numpy as np

PHI = (1.0 + 5.0 ** 0.5) / 2.0


def icosahedron():
    """Return (vertices (12,3) on the unit sphere, faces (20,3) int64, outward)."""
    verts = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            verts.append((0.0, s1, s2 * PHI))
            verts.append((s1, s2 * PHI, 0.0))
            verts.append((s2 * PHI, 0.0, s1))
    v = np.array(verts, dtype=np.float64)
    faces = []
    for i, j, k in itertools.combinations(range(12), 3):
        dij = np.linalg.norm(v[i] - v[j])
        djk = np.linalg.norm(v[j] - v[k])
        dik = np.linalg.norm(v[i] - v[k])
        if abs(dij - 2.0) < 1e-9 and abs(djk - 2.0) < 1e-9 and abs(dik - 2.0) < 1e-9:
            nrm = np.cross(v[j] - v[i], v[k] - v[i])
            if np.dot(nrm, v[i] + v[j] + v[k]) < 0.0:
                j, k = k, j
            faces.append((i, j, k))
    v = v / np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array(faces, dtype=np.int64)
    assert f.shape == (20, 3)
    return v, f


def refine(v, f, project=True):
    """One 1->4 refinement step.  Children of face (a,b,c) are, in order,
    (a,ab,ca), (ab,b,bc), (ca,bc,c), (ab,bc,ca); midpoints are shared between
    neighbouring faces and projected onto the unit sphere when `project`."""
    verts = [row for row in v]
    mid = {}

    def midpoint(i, j):
        key = (i, j) if i < j else (j, i)
        idx = mid.get(key)
        if idx is None:
            p = 0.5 * (v[i] + v[j])
            if project:
                p = p / np.linalg.norm(p)
            idx = len(verts)
            verts.append(p)
            mid[key] = idx
        return idx

    out = np.empty((4 * len(f), 3), dtype=np.int64)
    for t, (a, b, c) in enumerate(f):
        ab = midpoint(a, b)
        bc = midpoint(b, c)
        ca = midpoint(c, a)
        out[4 * t + 0] = (a, ab, ca)
        out[4 * t + 1] = (ab, b, bc)
        out[4 * t + 2] = (ca, bc, c)
        out[4 * t + 3] = (ab, bc, ca)
    return np.array(verts, dtype=np.float64), out


def icosphere(r):
    """Unit-sphere mesh refined r times: n = 20*4**r flat triangles."""
    v, f = icosahedron()
    for _ in range(r):
        v, f = refine(v, f, project=True)
    return v, f


def ellipsoid(r, axes):
    """Icosphere(r) with vertices scaled by axes=(ax, ay, az)."""
    v, f = icosphere(r)
    return v * np.asarray(axes, dtype=np.float64)[None, :], f


def triangle_data(v, f):
    """Centroids (n,3), areas (n,), per-triangle vertex bbox lo/hi (n,3)."""
    p0, p1, p2 = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    centroid = (p0 + p1 + p2) / 3.0
    area = 0.5 * np.linalg.norm(np.cross(p1 - p0, p2 - p0), axis=1)
    lo = np.minimum(np.minimum(p0, p1), p2)
    hi = np.maximum(np.maximum(p0, p1), p2)
    return centroid, area, lo, hi


def interval_cells(n):
    """The interval [0, 1] cut into n equal cells (the d = 1 problems of Sec. 6.1), embedded in
    R^3 on the x axis: (midpoints (n,3), lengths (n,), cell bbox lo/hi (n,3))."""
    x = np.linspace(0.0, 1.0, n + 1)
    z = np.zeros(n)
    lo = np.stack([x[:-1], z, z], axis=1)
    hi = np.stack([x[1:], z, z], axis=1)
    return 0.5 * (lo + hi), np.diff(x), lo, hi


def ellipse_panels(n, axes=(0.5, 0.5)):
    """A closed curve for the d = 2 problems of Sec. 6.1: the ellipse with semi-axes `axes`,
    cut into n straight panels between the points at angles 2 pi i / n, embedded in R^3 in the
    z = 0 plane: (panel midpoints (n,3), panel lengths (n,), panel bbox lo/hi (n,3)).  The
    default circle of radius 1/2 has logarithmic capacity 1/2 < 1, so the single-layer
    operator with kernel -log|x - y| / (2 pi) is positive definite on it."""
    t = 2.0 * np.pi * np.arange(n + 1) / n
    p = np.stack([axes[0] * np.cos(t), axes[1] * np.sin(t), np.zeros(n + 1)], axis=1)
    a, b = p[:-1], p[1:]
    return 0.5 * (a + b), np.linalg.norm(b - a, axis=1), np.minimum(a, b), np.maximum(a, b)
