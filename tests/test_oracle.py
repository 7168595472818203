"""Pins of the CPU oracle against what the mathematics fixes (CPU only):
hand-worked and library LU, Eckart-Young for rounded addition, the
untruncated limit (eps -> 0) and the all-dense structure (eta = 0), both of
which must reproduce the unique unpivoted dense LU, solve accuracy, the rank
invariant, and planted mistakes that these pins must catch."""
import numpy as np
import pytest
import scipy.linalg

from bem_inputs import build_problem
from oracle import HLUOracle, build_hmatrix, densify
from oracle.dense import lu_nopiv, solve_unit_lower, solve_upper, solve_upper_right
from oracle.errors import factor_error, lu_solve, solve_error
from oracle.hmatrix import hmul, hmul_t


def test_lu_hand_worked_2x2():
    a = np.array([[4.0, 2.0], [2.0, 3.0]])
    lu_nopiv(a)
    assert np.array_equal(a, np.array([[4.0, 2.0], [0.5, 2.0]]))


def test_lu_matches_scipy_without_pivoting():
    rng = np.random.default_rng(0)
    n = 40
    a = rng.standard_normal((n, n))
    a += np.diag(np.abs(a).sum(axis=0) + 1.0)  # column dominant: partial pivoting never swaps
    p, l, u = scipy.linalg.lu(a)
    assert np.array_equal(p, np.eye(n))
    f = a.copy()
    lu_nopiv(f)
    assert np.allclose(np.tril(f, -1) + np.eye(n), l, atol=1e-14)
    assert np.allclose(np.triu(f), u, atol=1e-12)


def test_triangular_solves_brute_force():
    rng = np.random.default_rng(1)
    n = 12
    a = rng.standard_normal((n, n)) + n * np.eye(n)
    f = a.copy()
    lu_nopiv(f)
    L = np.tril(f, -1) + np.eye(n)
    U = np.triu(f)
    x = rng.standard_normal((n, 3))
    assert np.allclose(L @ solve_unit_lower(f, x.copy()), x)
    assert np.allclose(U @ solve_upper(f, x.copy()), x)
    y = rng.standard_normal((3, n))
    assert np.allclose(solve_upper_right(f, y.copy()) @ U, y)


def test_rounded_addition_eckart_young(prob320):
    """T_eps(X) of X = Q1 diag(sigma) Q2^T given as two stacked factor pairs keeps
    exactly the sigma_i > eps*sigma_1 and leaves ||X - T(X)||_2 = sigma_{k+1}."""
    rng = np.random.default_rng(2)
    sig = np.array([1.0, 0.5, 1e-3, 5e-5, 1e-6])
    q1, _ = np.linalg.qr(rng.standard_normal((30, 5)))
    q2, _ = np.linalg.qr(rng.standard_normal((20, 5)))
    X = q1 @ np.diag(sig) @ q2.T
    # split X = U1 V1^T + U2 V2^T with non-orthogonal pieces
    g = rng.standard_normal((5, 5)) + 3 * np.eye(5)
    U1, V1 = q1 @ np.diag(sig) @ g[:, :3], q2 @ np.linalg.inv(g)[:3].T
    U2, V2 = q1 @ np.diag(sig) @ g[:, 3:], q2 @ np.linalg.inv(g)[3:].T
    o = HLUOracle(prob320, 1e-4)
    U, V = o.rounded_add(np.hstack([U1, U2]), np.hstack([V1, V2]))
    assert U.shape[1] == 3
    assert np.allclose(np.linalg.svd(U @ V.T, compute_uv=False)[:3], sig[:3], rtol=1e-10)
    assert np.isclose(np.linalg.norm(X - U @ V.T, 2), sig[3], rtol=1e-8)
    # a dense contribution enters in factorised form (identity on one side):
    # the result is the truncated SVD of the dense sum
    U, V = o.rounded_add(np.hstack([U1, X]), np.hstack([V1, np.eye(20)]))
    ref = np.linalg.svd(U1 @ V1.T + X, compute_uv=False)
    k = int(np.count_nonzero(ref > 1e-4 * ref[0]))
    assert U.shape[1] == k
    assert np.isclose(np.linalg.norm(U1 @ V1.T + X - U @ V.T, 2), ref[k], rtol=1e-8)


def _dense_lu_of(hm):
    a = densify(hm)
    f = a.copy()
    lu_nopiv(f)
    return a, f


def _check_vs_dense(p, eps_factor):
    hm = build_hmatrix(p)
    a, f = _dense_lu_of(hm)
    o = HLUOracle(p, eps_factor).factor()
    g = densify(o.A)
    return np.max(np.abs(g - f)) / np.max(np.abs(a)), o


def test_untruncated_limit_equals_dense_lu(prob1280):
    """eps -> 0: H-LU reproduces the unique unpivoted LU of the densified A_H
    (n = 1280 is the smallest sphere here with admissible blocks at eta = 2)."""
    assert np.count_nonzero(prob1280.kind == 1) > 0
    err, o = _check_vs_dense(prob1280, 1e-15)
    assert err < 1e-12
    assert o.c.min_pivot > 0.0


def test_all_dense_structure_equals_dense_lu():
    """eta = 0: no admissible block, the recursive structure is plain blocked LU."""
    p = build_problem(2, 32, 0.0, 1e-4, nrhs=1)
    assert np.all(p.kind == 0)
    err, _ = _check_vs_dense(p, 1e-4)
    assert err < 1e-13


def test_factor_and_solve_quality(prob1280):
    p = prob1280
    A = build_hmatrix(p)
    o = HLUOracle(p, p.eps).factor()
    assert o.c.min_pivot > 0.0  # A = K D with K SPD: all pivots positive
    efac = factor_error(A, o.A, p.n)
    assert efac <= 10 * p.eps
    x = lu_solve(o.A, p.b_perm())
    esol = solve_error(A, x, p.b_perm())
    assert np.all(esol <= 10 * p.eps)


def test_rank_invariant_every_truncation(prob1280):
    o = HLUOracle(prob1280, 1e-4)
    seen = []
    orig = o.rounded_add

    def checked(Us, Vs):
        U, V = orig(Us, Vs)
        seen.append((U.shape[1], Us.shape[0], Vs.shape[0]))
        return U, V
    o.rounded_add = checked
    o.factor()
    assert seen
    assert all(0 <= k <= min(m, n) for k, m, n in seen)
    for leaf in o.A.leaves():
        if leaf.kind == "lowrank":
            assert leaf.rank <= min(leaf.m, leaf.n)


def test_solve_untruncated_matches_dense_solve(prob1280):
    p = prob1280
    hm = build_hmatrix(p)
    a = densify(hm)
    o = HLUOracle(p, 1e-15).factor()
    x = lu_solve(o.A, p.b_perm())
    xd = np.linalg.solve(a, p.b_perm())
    assert np.max(np.abs(x - xd)) / np.max(np.abs(xd)) < 1e-11


def test_hmul_matches_dense(prob320):
    hm = build_hmatrix(prob320)
    a = densify(hm)
    x = np.random.default_rng(4).standard_normal((prob320.n, 3))
    assert np.allclose(hmul(hm, x), a @ x, rtol=1e-13, atol=1e-13)
    assert np.allclose(hmul_t(hm, x), a.T @ x, rtol=1e-13, atol=1e-13)


# ----------------------------------------------------------- planted mistakes
def _planted(monkeypatch, prob, attr, fn):
    monkeypatch.setattr(HLUOracle, attr, fn)
    err, _ = _check_vs_dense(prob, 1e-15)
    return err


def test_planted_dropped_schur_update_is_caught(prob320, monkeypatch):
    orig = HLUOracle.addmul

    def drop(self, C, alpha, A, B):
        if C.kind == "dense" and A.kind == "dense":
            return  # forget the dense x dense Schur contributions
        return orig(self, C, alpha, A, B)
    assert _planted(monkeypatch, prob320, "addmul", drop) > 1e-6


def test_planted_sign_error_is_caught(prob320, monkeypatch):
    orig = HLUOracle.addmul
    monkeypatch.setattr(HLUOracle, "addmul", lambda self, C, a, A, B: orig(self, C, -a, A, B))
    err, _ = _check_vs_dense(prob320, 1e-15)
    assert err > 1e-6


def test_planted_transposed_operand_is_caught(prob1280, monkeypatch):
    def wrong(self, U, X):
        if X.kind == "lowrank":
            self.trsm_l_panel(U, X.V)  # applies the lower factor to the wrong side
        else:
            return orig(self, U, X)
    orig = HLUOracle.trsm_u
    assert _planted(monkeypatch, prob1280, "trsm_u", wrong) > 1e-6


def test_planted_truncation_off_by_one_is_caught(prob320, monkeypatch):
    """Keeping one singular value too few must fail the Eckart-Young pin."""
    monkeypatch.setattr(HLUOracle, "_keep",
                        lambda self, sig: max(0, int(np.count_nonzero(sig > self.eps * sig[0])) - 1))
    with pytest.raises(AssertionError):
        test_rounded_addition_eckart_young(prob320)


@pytest.mark.parametrize("dim,eta", [(1, 0.25), (1, 1.0), (2, 0.5)])
def test_factor_quality_log_kernels(dim, eta):
    """The d = 1, 2 log-kernel problems of Sec. 6.1 with the eta values of Table 1: the oracle's
    factors and solve stay at the truncation level, as for the d = 3 problems."""
    p = build_problem(3, 32, eta, 1e-4, nrhs=1, dim=dim)
    assert (p.kind == 1).any() and (p.kind == 0).any()
    A = build_hmatrix(p)
    o = HLUOracle(p, p.eps).factor()
    assert o.c.min_pivot > 0.0
    assert factor_error(A, o.A, p.n) <= 10 * p.eps
    assert np.all(solve_error(A, lu_solve(o.A, p.b_perm()), p.b_perm()) <= 10 * p.eps)


# ------------------------------------------- the error estimator against dense norms
def _dense_factor_error(A, F):
    """||A_H - L U||_2 / ||A_H||_2 with every matrix formed densely (SVD-based 2-norms)."""
    a = densify(A)
    f = densify(F)
    L = np.tril(f, -1) + np.eye(a.shape[0])
    U = np.triu(f)
    return np.linalg.norm(a - L @ U, 2) / np.linalg.norm(a, 2)


def _estimator_cases():
    # n = 320 with leaf 16 (low-rank blocks at eta = 2, eps 1e-3) and the n = 1280 sphere at eps 1e-4
    return [build_problem(2, 16, 2.0, 1e-3, nrhs=1), build_problem(3, 32, 2.0, 1e-4, nrhs=1)]


@pytest.fixture(scope="module")
def estimator_cases():
    out = []
    for p in _estimator_cases():
        A = build_hmatrix(p)
        o = HLUOracle(p, p.eps).factor()
        out.append((p, A, o))
    return out


def test_factor_error_estimator_equals_dense_two_norm(estimator_cases):
    """The power-iteration E_fac (M = A_H - L U applied through the block structure, transposes by
    the transposed traversal) agrees with the 2-norms of the densified matrices to 1e-2."""
    for p, A, o in estimator_cases:
        ref = _dense_factor_error(A, o.A)
        assert ref > 1e-8  # a case with real truncation, not rounding noise
        est = factor_error(A, o.A, p.n)
        assert abs(est - ref) <= 1e-2 * ref, (p.n, est, ref)


def test_planted_missing_unit_diagonal_in_apply_lower_is_caught(estimator_cases, monkeypatch):
    import oracle.errors as oe
    orig = oe.apply_lower
    monkeypatch.setattr(oe, "apply_lower", lambda F, x: orig(F, x) - x)  # L without its unit diagonal
    p, A, o = estimator_cases[1]
    ref = _dense_factor_error(A, o.A)
    assert abs(factor_error(A, o.A, p.n) - ref) > 1e-2 * ref


def test_planted_untransposed_apply_upper_t_is_caught(estimator_cases, monkeypatch):
    import oracle.errors as oe
    monkeypatch.setattr(oe, "apply_upper_t", lambda F, x: oe.apply_upper(F, x))  # U instead of U^T
    p, A, o = estimator_cases[1]
    ref = _dense_factor_error(A, o.A)
    assert abs(factor_error(A, o.A, p.n) - ref) > 1e-2 * ref


# ----------------------------------------------- the plain definition of addmul
def test_plain_reading_meets_the_bound_and_agrees_untruncated(prob1280):
    """The plain definition (the exact product formed densely, one truncated SVD of the exact sum per
    low-rank target leaf) and the split/merge reading both meet E_fac <= 10 eps at n = 1280, and at
    eps -> 0 both reproduce the unique unpivoted LU, so they agree to rounding."""
    p = prob1280
    A = build_hmatrix(p)
    res = {}
    for reading in ("split", "plain"):
        o = HLUOracle(p, p.eps, reading=reading).factor()
        assert o.c.min_pivot > 0.0
        assert _dense_factor_error(A, o.A) <= 10 * p.eps
        assert factor_error(A, o.A, p.n) <= 10 * p.eps
        res[reading] = densify(HLUOracle(p, 1e-15, reading=reading).factor().A)
    scale = np.max(np.abs(densify(A)))
    assert np.max(np.abs(res["split"] - res["plain"])) <= 1e-12 * scale
    assert HLUOracle(p, p.eps, reading="plain").factor().c.events["prod_dense_exact"] > 0


def test_dense_truncation_eckart_young(prob320):
    """truncate_dense (the plain rounded addition) keeps exactly sigma_i > eps sigma_1 of a block with
    known singular values and leaves ||X - T(X)||_2 = sigma_{k+1}."""
    rng = np.random.default_rng(5)
    sig = np.array([2.0, 0.3, 4e-4, 1e-4, 3e-7])
    q1, _ = np.linalg.qr(rng.standard_normal((25, 5)))
    q2, _ = np.linalg.qr(rng.standard_normal((18, 5)))
    X = q1 @ np.diag(sig) @ q2.T
    o = HLUOracle(prob320, 1e-4, reading="plain")
    U, V = o.truncate_dense(X)
    assert U.shape[1] == 3  # 1e-4 * 2 = 2e-4 < 4e-4 kept, 1e-4 dropped
    assert np.isclose(np.linalg.norm(X - U @ V.T, 2), sig[3], rtol=1e-8)
