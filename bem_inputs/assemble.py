"""Matrix entries and leaf data of the BEM H-matrix.

Kernels: the Laplace kernels of Sec. 6.1 in collocation form, one element
(centroid c_i, size a_i: area of a flat triangle in d = 3, length of a cell or
straight panel in d = 1, 2) per degree of freedom:

    A_ij = a_j g(c_i, c_j)   (i != j),   g = 1 / (4 pi |x - y|)      (d = 3)
                                         g = -log|x - y|             (d = 1)
                                         g = -log|x - y| / (2 pi)    (d = 2)

and the self-term A_ii = the potential at c_i of the element itself with unit
density: sqrt(a_i / pi) / 2 for d = 3 (a flat disc of area a_i), and
a_i (1 - log(a_i / 2)) (d = 1) or that over 2 pi (d = 2), the exact integral of
-log|t| over |t| <= a_i / 2 (a straight element of length a_i centred at c_i).

Low-rank leaves (Sec. 3.1, "Low-rank blocks": X = A B^*): built by adaptive
cross approximation with partial pivoting and then recompressed by an SVD of
the small factor product, as the paper recompresses its interpolation factors
(Sec. 6.1).  The recompression keeps singular values sigma_i > eps * sigma_1.
ACA itself is the generator's choice of compression (the paper interpolates).

Storage per leaf (consumed as plain data by every solver): dense leaves as an
m x n column-major array; low-rank leaves as U (m x k) followed by V (n x k),
both column-major, representing U V^T.
"""
from __future__ import annotations

import numpy as np

FOUR_PI = 4.0 * np.pi


def _g(r, dim):
    """Kernel value at distance r > 0."""
    if dim == 3:
        return 1.0 / (FOUR_PI * r)
    if dim == 1:
        return -np.log(r)
    if dim == 2:
        return -np.log(r) / (2.0 * np.pi)
    raise ValueError(f"dim must be 1, 2 or 3, got {dim}")


def self_term(a, dim):
    """A_ii for elements of size a (see the module docstring)."""
    if dim == 3:
        return np.sqrt(a / np.pi) / 2.0
    s = a * (1.0 - np.log(0.5 * a))
    return s if dim == 1 else s / (2.0 * np.pi)


def kernel_block(centroid, area, rows, cols, dim=3):
    """Dense kernel block A[rows][:, cols] (original DoF indices)."""
    d = centroid[rows][:, None, :] - centroid[cols][None, :, :]
    r = np.sqrt(np.einsum("ijk,ijk->ij", d, d))
    same = rows[:, None] == cols[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        out = area[cols][None, :] * _g(r, dim)
    if same.any():
        ii, jj = np.nonzero(same)
        out[ii, jj] = self_term(area[rows[ii]], dim)
    return out


def _kernel_row(centroid, area, i, cols, dim=3):
    d = centroid[cols] - centroid[i]
    return area[cols] * _g(np.sqrt(np.einsum("ij,ij->i", d, d)), dim)


def _kernel_col(centroid, area, rows, j, dim=3):
    d = centroid[rows] - centroid[j]
    return area[j] * _g(np.sqrt(np.einsum("ij,ij->i", d, d)), dim)


def aca_partial(centroid, area, rows, cols, eps, dim=3):
    """ACA with partial pivoting on an admissible block (rows, cols disjoint).

    Start row: local row 0.  Column pivot: argmax |residual row| (lowest index
    on ties).  Next row: argmax |residual column| over unused rows.  Stops when
    |u_k| |v_k| <= 0.1 * eps * |S_k|_F (|S_k|_F updated incrementally) or when
    k reaches min(m, n).  Returns U (m x k), V (n x k) with block ~= U V^T.
    """
    m, n = len(rows), len(cols)
    kmax = min(m, n)
    U = np.zeros((m, kmax))
    V = np.zeros((n, kmax))
    used = np.zeros(m, dtype=bool)
    i = 0
    k = 0
    s2 = 0.0
    while k < kmax:
        row = _kernel_row(centroid, area, rows[i], cols, dim)
        if k:
            row -= V[:, :k] @ U[i, :k]
        used[i] = True
        j = int(np.argmax(np.abs(row)))
        if row[j] == 0.0:
            free = np.flatnonzero(~used)
            if free.size == 0:
                break
            i = int(free[0])
            continue
        v = row / row[j]
        u = _kernel_col(centroid, area, rows, cols[j], dim)
        if k:
            u -= U[:, :k] @ V[j, :k]
            s2 += 2.0 * float(np.dot(U[:, :k].T @ u, V[:, :k].T @ v))
        uu, vv = float(u @ u), float(v @ v)
        s2 += uu * vv
        U[:, k] = u
        V[:, k] = v
        k += 1
        if np.sqrt(uu * vv) <= 0.1 * eps * np.sqrt(max(s2, 0.0)):
            break
        au = np.abs(u)
        au[used] = -1.0
        i = int(np.argmax(au))
        if au[i] < 0.0:
            break
    return U[:, :k], V[:, :k]


def recompress(U, V, eps):
    """SVD recompression of U V^T keeping sigma_i > eps*sigma_1; Sigma goes into U."""
    if U.shape[1] == 0:
        return U, V
    q1, r1 = np.linalg.qr(U)
    q2, r2 = np.linalg.qr(V)
    x, sig, yt = np.linalg.svd(r1 @ r2.T)
    if sig[0] == 0.0:
        return U[:, :0], V[:, :0]
    k = int(np.count_nonzero(sig > eps * sig[0]))
    return q1 @ (x[:, :k] * sig[:k]), q2 @ yt[:k].T
