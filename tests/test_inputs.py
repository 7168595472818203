"""Pins of the seeded input generator against closed forms of potential theory
and of the mesh construction (CPU only)."""
import numpy as np
import pytest

from bem_inputs import build_problem, icosphere, kernel_block, triangle_data
from bem_inputs.trees import admissible


@pytest.mark.parametrize("r", [0, 1, 2, 3])
def test_icosphere_counts_and_area(r):
    v, f = icosphere(r)
    assert f.shape[0] == 20 * 4 ** r
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0)
    _, area, _, _ = triangle_data(v, f)
    assert np.all(area > 0)
    assert area.sum() < 4 * np.pi
    # Euler characteristic of a closed genus-0 surface: V - E + F = 2
    edges = {tuple(sorted(e)) for t in f for e in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0]))}
    assert v.shape[0] - len(edges) + f.shape[0] == 2


def test_area_increases_to_4pi():
    tot = []
    for r in range(5):
        v, f = icosphere(r)
        tot.append(triangle_data(v, f)[1].sum())
    assert all(a < b for a, b in zip(tot, tot[1:]))
    # the inscribed polyhedron's area deficit is O(h^2): it shrinks 4x per refinement
    d = [4 * np.pi - a for a in tot]
    ratios = [d[i + 1] / d[i] for i in range(2, 4)]
    assert all(0.24 < q < 0.27 for q in ratios)


def _dense(r):
    v, f = icosphere(r)
    c, a, _, _ = triangle_data(v, f)
    idx = np.arange(c.shape[0])
    return kernel_block(c, a, idx, idx), c


def test_single_layer_closed_forms():
    """On the unit sphere the single-layer operator maps 1 -> 1 and the degree-1
    harmonic x -> x/3 (eigenvalue 1/(2l+1)); the collocation matrix reproduces
    both with an error that shrinks under refinement."""
    errs1, errsx = [], []
    for r in (2, 3):
        A, c = _dense(r)
        errs1.append(np.max(np.abs(A.sum(axis=1) - 1.0)))
        errsx.append(np.max(np.abs(A @ c[:, 0] - c[:, 0] / 3.0)))
    assert errs1[-1] < 0.05 and errs1[1] < errs1[0]
    assert errsx[-1] < 0.03 and errsx[1] < errsx[0]
    A, _ = _dense(3)
    x = np.linalg.solve(A, np.ones(A.shape[0]))
    assert np.max(np.abs(x - 1.0)) < 0.05


def test_matrix_is_kernel_times_area():
    """A = K D with K symmetric (1/(4 pi r), disc self-term) and D = diag(area)."""
    v, f = icosphere(2)
    c, a, _, _ = triangle_data(v, f)
    idx = np.arange(c.shape[0])
    A = kernel_block(c, a, idx, idx)
    K = A / a[None, :]
    assert np.allclose(K, K.T, rtol=1e-14, atol=0)
    assert np.all(np.linalg.eigvalsh(K) > 0)  # 1/|x| is a positive-definite kernel


def test_cluster_tree_partition(prob1280):
    t = prob1280.tree
    assert sorted(t.perm.tolist()) == list(range(prob1280.n))
    for c in range(t.n_clusters):
        if t.son0[c] >= 0:
            s0, s1 = t.son0[c], t.son1[c]
            assert t.begin[s0] == t.begin[c]
            assert t.begin[s1] == t.begin[c] + t.size[s0]
            assert t.size[s0] + t.size[s1] == t.size[c]
            assert t.size[c] > prob1280.leaf
        else:
            assert t.size[c] <= prob1280.leaf


def test_block_leaves_tile_matrix(prob1280):
    p = prob1280
    cover = np.zeros((p.n, p.n), dtype=np.int32)
    for l in range(p.n_leaves):
        r0, m, c0, n = p.leaf_ranges(l)
        cover[r0:r0 + m, c0:c0 + n] += 1
        if p.kind[l] == 1:
            assert r0 != c0  # never a diagonal block
            assert 0 <= p.rank[l] <= min(m, n)
    assert np.all(cover == 1)


def test_admissible_definition(prob1280):
    t = prob1280.tree
    # touching / overlapping boxes are never admissible
    assert not admissible(t, 0, 0, 2.0)
    for l in range(prob1280.n_leaves):
        if prob1280.kind[l] == 1:
            a, b = prob1280.row_cl[l], prob1280.col_cl[l]
            assert min(t.diam(a), t.diam(b)) <= 2.0 * t.dist(a, b)


def test_hmatrix_approximates_dense(prob1280):
    """||A_H x - A x|| / ||A x|| is of the order of the compression eps."""
    p = prob1280
    A, _ = _dense(3)
    Ap = A[np.ix_(p.tree.perm, p.tree.perm)]
    AH = np.zeros_like(Ap)
    for l in range(p.n_leaves):
        r0, m, c0, n = p.leaf_ranges(l)
        if p.kind[l] == 0:
            AH[r0:r0 + m, c0:c0 + n] = p.leaf_dense(l)
        else:
            U, V = p.leaf_factors(l)
            AH[r0:r0 + m, c0:c0 + n] = U @ V.T
    x = np.random.default_rng(3).standard_normal(p.n)
    rel = np.linalg.norm(AH @ x - Ap @ x) / np.linalg.norm(Ap @ x)
    assert rel < 3 * p.eps
    assert np.linalg.norm(AH - Ap, 2) / np.linalg.norm(Ap, 2) < 10 * p.eps


def test_rhs_is_seeded_normal(prob320):
    b = np.random.default_rng(0).standard_normal((2, prob320.n)).T
    assert np.array_equal(prob320.b, b)


@pytest.mark.parametrize("dim", [1, 2])
def test_log_kernel_entries_and_self_term(dim):
    """d = 1, 2 (Sec. 6.1): off-diagonal entries a_j g(c_i, c_j) with g = -log r (d = 1) or
    -log r / (2 pi) (d = 2); the self-term equals the integral of g over the element itself,
    computed here by adaptive quadrature (scipy) of -log|t| on both halves."""
    from scipy.integrate import quad
    from bem_inputs.mesh import ellipse_panels, interval_cells
    c, a, lo, hi = interval_cells(40) if dim == 1 else ellipse_panels(40)
    idx = np.arange(40)
    A = kernel_block(c, a, idx, idx, dim)
    scale = 1.0 if dim == 1 else 1.0 / (2 * np.pi)
    i, j = 3, 17
    assert np.isclose(A[i, j], -a[j] * np.log(np.linalg.norm(c[i] - c[j])) * scale, rtol=1e-14)
    h = a[5]
    half = quad(lambda t: -np.log(t), 0.0, h / 2)[0]
    assert np.isclose(A[5, 5], 2 * half * scale, rtol=1e-10)
    assert np.all(lo <= c) and np.all(c <= hi)


def test_curve_and_interval_geometry():
    from bem_inputs.mesh import ellipse_panels, interval_cells
    c, a, _, _ = interval_cells(64)
    assert np.isclose(a.sum(), 1.0) and np.allclose(c[:, 1:], 0.0)
    # inscribed polygon of the circle of radius 1/2: perimeter -> pi from below, O(1/n^2)
    p1 = ellipse_panels(64)[1].sum()
    p2 = ellipse_panels(128)[1].sum()
    assert p1 < p2 < np.pi
    assert np.isclose((np.pi - p1) / (np.pi - p2), 4.0, rtol=1e-2)
