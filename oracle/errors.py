"""Applying the H-LU factors and measuring their quality (test infrastructure only).

solve:  L y = b (unit lower, forward), then U x = y (backward), through the
        block structure: for a partitioned diagonal block the off-diagonal
        sons act as exact H x dense products (Sec. 3.1, y = U (V^T z) on
        low-rank leaves).
E_fac:  ||A_H - L U||_2 / ||A_H||_2, both norms by power iteration on M^T M,
        M applied only through matrix-vector products.
E_sol:  ||b - A_H x||_2 / ||b||_2 per column.
"""
from __future__ import annotations

import numpy as np

from .dense import solve_unit_lower, solve_upper
from .hmatrix import hmul, hmul_t


def solve_lower(F, y):
    """y := L^{-1} y in place (L: unit lower part of the factored block F)."""
    if F.kind == "dense":
        solve_unit_lower(F.D, y)
        return y
    (f00, _), (f10, f11) = F.sons
    m0 = f00.m
    solve_lower(f00, y[:m0])
    y[m0:] -= hmul(f10, y[:m0])
    solve_lower(f11, y[m0:])
    return y


def solve_upper_h(F, y):
    """y := U^{-1} y in place (U: upper part of the factored block F)."""
    if F.kind == "dense":
        solve_upper(F.D, y)
        return y
    (f00, f01), (_, f11) = F.sons
    m0 = f00.m
    solve_upper_h(f11, y[m0:])
    y[:m0] -= hmul(f01, y[m0:])
    solve_upper_h(f00, y[:m0])
    return y


def lu_solve(F, b_perm):
    """x = U^{-1} L^{-1} b for b in cluster order (copy)."""
    y = np.array(b_perm, dtype=np.float64, copy=True)
    solve_lower(F, y)
    solve_upper_h(F, y)
    return y


def apply_upper(F, x):
    if F.kind == "dense":
        return np.triu(F.D) @ x
    (f00, f01), (_, f11) = F.sons
    m0 = f00.m
    out = np.empty_like(x)
    out[:m0] = apply_upper(f00, x[:m0]) + hmul(f01, x[m0:])
    out[m0:] = apply_upper(f11, x[m0:])
    return out


def apply_lower(F, x):
    if F.kind == "dense":
        return np.tril(F.D, -1) @ x + x
    (f00, _), (f10, f11) = F.sons
    m0 = f00.m
    out = np.empty_like(x)
    out[:m0] = apply_lower(f00, x[:m0])
    out[m0:] = hmul(f10, x[:m0]) + apply_lower(f11, x[m0:])
    return out


def apply_upper_t(F, x):
    if F.kind == "dense":
        return np.triu(F.D).T @ x
    (f00, f01), (_, f11) = F.sons
    m0 = f00.m
    out = np.empty_like(x)
    out[:m0] = apply_upper_t(f00, x[:m0])
    out[m0:] = hmul_t(f01, x[:m0]) + apply_upper_t(f11, x[m0:])
    return out


def apply_lower_t(F, x):
    if F.kind == "dense":
        return np.tril(F.D, -1).T @ x + x
    (f00, _), (f10, f11) = F.sons
    m0 = f00.m
    out = np.empty_like(x)
    out[:m0] = apply_lower_t(f00, x[:m0]) + hmul_t(f10, x[m0:])
    out[m0:] = apply_lower_t(f11, x[m0:])
    return out


def power_norm(apply, apply_t, n, seed=1, iters=30, rtol=1e-3):
    """||M||_2 by power iteration on M^T M; start vector N(0,1) from `seed`."""
    x = np.random.default_rng(seed).standard_normal(n)
    x /= np.linalg.norm(x)
    lam_old = 0.0
    lam = 0.0
    for _ in range(iters):
        z = apply_t(apply(x))
        lam = float(np.linalg.norm(z))
        if lam == 0.0:
            return 0.0
        x = z / lam
        if lam_old and abs(lam - lam_old) <= rtol * lam:
            break
        lam_old = lam
    return float(np.sqrt(lam))


def factor_error(A, F, n, seed=1):
    """E_fac = ||A_H - L U||_2 / ||A_H||_2 for the original H-matrix A and factors F."""
    def m_apply(x):
        return hmul(A, x) - apply_lower(F, apply_upper(F, x))

    def m_apply_t(x):
        return hmul_t(A, x) - apply_upper_t(F, apply_lower_t(F, x))

    num = power_norm(m_apply, m_apply_t, n, seed)
    den = power_norm(lambda x: hmul(A, x), lambda x: hmul_t(A, x), n, seed)
    return num / den


def solve_error(A, x, b):
    """Per-column ||b - A_H x|| / ||b|| (cluster order)."""
    r = b - hmul(A, x)
    return np.linalg.norm(r, axis=0) / np.linalg.norm(b, axis=0)
