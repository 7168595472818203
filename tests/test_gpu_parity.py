"""GPU parity: the CUDA H-LU through the C ABI against the CPU oracle on the
same seeded problems.

Tolerances.  Both sides run the same algorithm (same recursion, same
truncation points), so results agree to rounding unless a singular value lies
at the truncation threshold eps * sigma_1, where one side may keep it and the
other drop it; the two factors then differ by at most about eps times that
block's norm.  Hence: when every rank agrees, densified factors must agree to
1e-10 * max|A_H| (FP64 rounding after propagation through the recursion);
otherwise at most a handful of ranks may differ and the factors must agree to
10 * eps * max|A_H|.  Quality bounds are the ones fixed for the method:
E_fac = ||A_H - LU||_2 / ||A_H||_2 <= 10 eps and the solve error within 2x the
oracle's.
"""
import numpy as np
import pytest

from bem_inputs import build_problem
from oracle import HLUOracle, build_hmatrix, densify
from oracle.dense import lu_nopiv
from oracle.errors import factor_error, lu_solve, solve_error
from oracle.hmatrix import hmul

from gpu_helpers import factors_as_problem, gpu_factor, rank_agreement

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_1906_00874_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _to_orig(p, x_perm):
    x = np.empty_like(x_perm)
    x[p.tree.perm] = x_perm
    return x


def _dev(a):
    from paper_1906_00874_gb300.hlu import to_device_panel
    return to_device_panel(a)


def _check_factor_parity(p, h, o):
    q = factors_as_problem(p, h)
    same, tot = rank_agreement(o, q)
    amax = np.max(np.abs(densify(build_hmatrix(p))))
    err = np.max(np.abs(densify(build_hmatrix(q)) - densify(o.A))) / amax
    if same == tot:
        assert err <= 1e-10, err
    else:
        assert tot - same <= max(2, tot // 500), (same, tot)
        assert err <= 10 * p.eps, err
    return q, err, same, tot


@pytest.fixture(scope="module")
def case1280():
    p = build_problem(3, 32, 2.0, 1e-4, nrhs=3)
    o = HLUOracle(p, p.eps).factor()
    return p, o


def test_factor_parity_1280(case1280):
    p, o = case1280
    h = gpu_factor(p)
    q, err, same, tot = _check_factor_parity(p, h, o)
    A = build_hmatrix(p)
    assert factor_error(A, build_hmatrix(q), p.n) <= 10 * p.eps
    st = h.stats()
    assert st["max_rank"] <= 32
    h.close()


def test_solve_parity_1280(case1280):
    p, o = case1280
    h = gpu_factor(p)
    b = _dev(p.b)
    h.solve(b)
    x = b.cpu().numpy()
    xo = _to_orig(p, lu_solve(o.A, p.b_perm()))
    assert np.max(np.abs(x - xo)) / np.max(np.abs(xo)) <= 1e-10
    A = build_hmatrix(p)
    e_gpu = solve_error(A, x[p.tree.perm], p.b_perm())
    e_or = solve_error(A, xo[p.tree.perm], p.b_perm())
    assert np.all(e_gpu <= 2 * e_or)
    h.close()


def test_matvec_parity_1280(case1280):
    p, _ = case1280
    from paper_1906_00874_gb300 import HLU
    import torch
    h = HLU.from_problem(p)
    x = np.random.default_rng(7).standard_normal((p.n, 5))
    xd = _dev(x)
    yd = _dev(np.zeros_like(x))
    h.matvec(xd, yd)
    y = yd.cpu().numpy()
    yo = _to_orig(p, hmul(build_hmatrix(p), x[p.tree.perm]))
    assert np.max(np.abs(y - yo)) / np.max(np.abs(yo)) <= 1e-13
    torch.cuda.synchronize()
    h.close()


def test_factor_parity_5120():
    p = build_problem(4, 32, 2.0, 1e-4, nrhs=1)
    o = HLUOracle(p, p.eps).factor()
    h = gpu_factor(p)
    q, err, same, tot = _check_factor_parity(p, h, o)
    b = _dev(p.b)
    h.solve(b)
    A = build_hmatrix(p)
    xo = lu_solve(o.A, p.b_perm())
    e_gpu = solve_error(A, b.cpu().numpy()[p.tree.perm], p.b_perm())
    assert np.all(e_gpu <= 2 * solve_error(A, xo, p.b_perm()))
    h.close()


@pytest.mark.parametrize("dim,eta", [(1, 0.25), (1, 1.0), (2, 0.5)])
def test_factor_parity_log_kernels(dim, eta):
    """d = 1, 2 log-kernel problems (Sec. 6.1) with the eta values of Table 1: factors equal
    the oracle's, and the GPU solve is as accurate as the oracle's."""
    p = build_problem(3, 32, eta, 1e-4, nrhs=2, dim=dim)
    o = HLUOracle(p, p.eps).factor()
    h = gpu_factor(p)
    _check_factor_parity(p, h, o)
    b = _dev(p.b)
    h.solve(b)
    A = build_hmatrix(p)
    xo = lu_solve(o.A, p.b_perm())
    e_gpu = solve_error(A, b.cpu().numpy()[p.tree.perm], p.b_perm())
    assert np.all(e_gpu <= 2 * solve_error(A, xo, p.b_perm()))
    h.close()


@pytest.mark.parametrize("inv_block", [-1, 64, 256, 2048])
def test_inverse_block_solve_equals_substitution(case1280, inv_block):
    """The solve by inverse blocks (the diagonal blocks of order <= inv_block inverted at the end of
    the factorisation and applied as products) gives the oracle's block substitution; -1 is the
    plain substitution.  The factors do not depend on it."""
    p, o = case1280
    h = gpu_factor(p, inv_block=inv_block)
    _check_factor_parity(p, h, o)
    b = _dev(p.b)
    h.solve(b)
    xo = _to_orig(p, lu_solve(o.A, p.b_perm()))
    assert np.max(np.abs(b.cpu().numpy() - xo)) / np.max(np.abs(xo)) <= 1e-10
    h.close()


def test_all_dense_structure_is_dense_lu():
    """eta = 0: every block dense; the GPU result is the unique unpivoted LU."""
    p = build_problem(3, 32, 0.0, 1e-4, nrhs=1)
    h = gpu_factor(p)
    q = factors_as_problem(p, h)
    a = densify(build_hmatrix(p))
    f = a.copy()
    lu_nopiv(f)
    assert np.max(np.abs(densify(build_hmatrix(q)) - f)) / np.max(np.abs(a)) <= 1e-12
    h.close()


def test_repeat_factor_is_deterministic(case1280):
    p, _ = case1280
    h = gpu_factor(p)
    r1 = h.get_factors()
    h.factor(p.eps)
    r2 = h.get_factors()
    assert np.array_equal(r1[0], r2[0]) and np.array_equal(r1[2], r2[2])
    h.close()


def test_solve_chunks_and_leading_dimension(case1280):
    """nrhs wider than one solve pass, and ld > n, give the column-by-column result."""
    import torch
    p, _ = case1280
    h = gpu_factor(p, nrhs_max=4)
    B = np.random.default_rng(11).standard_normal((p.n, 9))
    big = torch.zeros((p.n + 7, 9), dtype=torch.float64, device="cuda")
    big[: p.n] = torch.tensor(B, device="cuda")
    view = big.t().contiguous().t()[: p.n]  # column-major, ld = n + 7
    assert view.stride(1) == p.n + 7
    h.solve(view)
    X = view.cpu().numpy()
    for j in (0, 4, 8):
        bj = _dev(B[:, j].copy())
        h.solve(bj)
        assert np.max(np.abs(bj.cpu().numpy() - X[:, j])) <= 1e-12 * np.max(np.abs(X[:, j]))
    h.close()


def test_zero_rhs_and_state_errors(case1280):
    import torch
    from paper_1906_00874_gb300 import HLU, HLUError
    p, _ = case1280
    h = HLU.from_problem(p)
    b = _dev(p.b)
    with pytest.raises(HLUError) as e:
        h.solve(b)
    assert e.value.status == 3  # HLU_ESTATE: solve before factor
    h.factor(p.eps)
    empty = torch.zeros((p.n, 0), dtype=torch.float64, device="cuda")
    h.solve(empty)
    h.close()


def test_fp32_factor_is_a_good_preconditioner(case1280):
    """FP32 factors: E_fac stays at the truncation level (FP32 rounding ~6e-8 is
    far below eps = 1e-4); FP64 iterative refinement reaches 1e-10."""
    import torch
    from paper_1906_00874_gb300 import HLU, HLU_FP32
    p, _ = case1280
    h = HLU.from_problem(p, precision=HLU_FP32)
    h.factor(p.eps)
    q = factors_as_problem(p, h)
    A = build_hmatrix(p)
    assert factor_error(A, build_hmatrix(q), p.n) <= 10 * p.eps
    b = _dev(p.b)
    x = torch.zeros_like(b)
    r = b.clone()
    ax = torch.zeros_like(b)
    bn = torch.linalg.norm(b, dim=0)
    for it in range(12):
        d = r.clone()
        h.solve(d)
        x += d
        h.matvec(x, ax)
        r = b - ax
        res = (torch.linalg.norm(r, dim=0) / bn).max().item()
        if res <= 1e-10:
            break
    assert res <= 1e-10 and it <= 6
    # the residual is checked independently with the oracle's H-matvec
    xr = x.cpu().numpy()[p.tree.perm]
    assert np.all(solve_error(A, xr, p.b_perm()) <= 2e-10)
    h.close()


def test_solve_refined_matches_manual_refinement(case1280):
    """The library's refinement loop gives the same iterate as the loop written
    with hlu_solve + hlu_matvec, and reaches the tolerance."""
    import torch
    from paper_1906_00874_gb300 import HLU, HLU_FP32
    p, _ = case1280
    h = HLU.from_problem(p, precision=HLU_FP32)
    h.factor(p.eps)
    b = _dev(p.b)
    x = torch.zeros_like(b)
    it, res = h.solve_refined(b, x, tol=1e-10, max_iter=20)
    assert res <= 1e-10
    xm = torch.zeros_like(b)
    r = b.clone()
    ax = torch.zeros_like(b)
    for _ in range(it):
        d = r.clone()
        h.solve(d)
        xm += d
        h.matvec(xm, ax)
        r = b - ax
    assert torch.max(torch.abs(xm - x)).item() <= 1e-12 * torch.max(torch.abs(x)).item()
    st = h.stats()
    assert st["solve_flops"] > 0 and st["model_flops"] > 0
    h.close()


@pytest.mark.parametrize("n", [1, 2, 127])
@pytest.mark.parametrize("inv_block", [-1, 0])
def test_single_dense_leaf_degenerate_sizes(n, inv_block):
    """Degenerate H-matrices: one dense leaf of order 1, 2 or 127 (no low-rank block, one task of each
    kind).  The factorisation is the unpivoted LU (oracle), the solve the dense solve."""
    from paper_1906_00874_gb300 import HLU
    g = np.random.default_rng(n)
    a = g.standard_normal((n, n)) + 2.0 * n * np.eye(n)
    b = g.standard_normal((n, 3))
    h = HLU(n, np.arange(n), [0], [n], [-1], [-1], [0], [0], [0], [0], [0], a.ravel(order="F"), inv_block=inv_block)
    h.factor(1e-4)
    _, _, data = h.get_factors()
    f = a.copy()
    lu_nopiv(f)
    assert np.max(np.abs(data[:n * n].reshape((n, n), order="F") - f)) <= 1e-13 * np.max(np.abs(f))
    bd = _dev(b)
    h.solve(bd)
    x = np.linalg.solve(a, b)
    assert np.max(np.abs(bd.cpu().numpy() - x)) <= 1e-12 * np.max(np.abs(x))
    h.close()
