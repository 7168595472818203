"""Dense building blocks of the H-LU (Sec. 3.1, "Dense blocks"): LU without
pivoting (L unit lower, U upper, both overwriting A; the unit diagonal of L is
not stored), and the two triangular solves.  Test infrastructure only.
"""
from __future__ import annotations

import numpy as np


def lu_nopiv(a):
    """In-place right-looking LU without pivoting of a square FP64 array.

    After the call the strict lower triangle holds L (unit diagonal implied)
    and the upper triangle holds U.  Returns the pivots u_kk.
    """
    m = a.shape[0]
    assert a.shape == (m, m)
    for k in range(m):
        piv = a[k, k]
        a[k + 1:, k] /= piv
        a[k + 1:, k + 1:] -= np.outer(a[k + 1:, k], a[k, k + 1:])
    return np.diag(a).copy()


def solve_unit_lower(lu, x):
    """x := L^{-1} x with L the unit lower triangle stored in `lu` (in place)."""
    m = lu.shape[0]
    for i in range(1, m):
        x[i] -= lu[i, :i] @ x[:i]
    return x


def solve_upper(lu, x):
    """x := U^{-1} x with U the upper triangle of `lu` (in place)."""
    m = lu.shape[0]
    for i in range(m - 1, -1, -1):
        if i + 1 < m:
            x[i] -= lu[i, i + 1:] @ x[i + 1:]
        x[i] /= lu[i, i]
    return x


def solve_upper_right(lu, x):
    """x := x U^{-1} (x has U's order as its column count), in place."""
    m = lu.shape[0]
    for j in range(m):
        if j:
            x[:, j] -= x[:, :j] @ lu[:j, j]
        x[:, j] /= lu[j, j]
    return x


def solve_unit_lower_right(lu, x):
    """x := x L^{-1} with L unit lower (used by transposed solves), in place."""
    m = lu.shape[0]
    for j in range(m - 2, -1, -1):
        x[:, j] -= x[:, j + 1:] @ lu[j + 1:, j]
    return x
