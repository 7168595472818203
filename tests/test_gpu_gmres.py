"""GPU GMRES(m) (hlu_solve_gmres): FP64 Krylov iteration on the original
H-matrix, right-preconditioned by the H-LU solve.

The iterate after k Arnoldi steps is pinned against a plain NumPy GMRES
written here (modified Gram-Schmidt, least squares by numpy.linalg.lstsq) with
the same preconditioner (the GPU solve) and the oracle's FP64 H-matvec; the
final residual is checked with the oracle's H-matvec as well.
"""
import numpy as np
import pytest

from bem_inputs import build_problem
from oracle import build_hmatrix
from oracle.errors import solve_error
from oracle.hmatrix import hmul

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_1906_00874_gb300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def prob():
    return build_problem(3, 32, 2.0, 1e-4, nrhs=3)


def _dev(a):
    from paper_1906_00874_gb300.hlu import to_device_panel
    return to_device_panel(a)


def _handle(p, precision):
    from paper_1906_00874_gb300 import HLU
    h = HLU.from_problem(p, precision=precision)
    h.factor(p.eps)
    return h


def _numpy_gmres(apply_a, apply_m, b, k):
    """k steps of right-preconditioned GMRES from x = 0 for one column (textbook form)."""
    beta = np.linalg.norm(b)
    V = [b / beta]
    Z = []
    H = np.zeros((k + 1, k))
    for j in range(k):
        Z.append(apply_m(V[j]))
        w = apply_a(Z[j])
        for i in range(j + 1):
            H[i, j] = V[i] @ w
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        V.append(w / H[j + 1, j])
    e1 = np.zeros(k + 1)
    e1[0] = beta
    y = np.linalg.lstsq(H, e1, rcond=None)[0]
    return sum(y[i] * Z[i] for i in range(k))


def test_gmres_iterate_matches_numpy_gmres(prob):
    """After exactly k = 3 Arnoldi steps the GPU iterate equals the textbook GMRES
    iterate built from the same preconditioner and the oracle's H-matvec."""
    import torch
    from paper_1906_00874_gb300 import HLU_FP32
    p = prob
    h = _handle(p, HLU_FP32)
    A = build_hmatrix(p)
    perm = p.tree.perm

    def apply_m(v):  # original order in and out, through the GPU solve (the preconditioner)
        d = _dev(v[:, None].copy())
        h.solve(d)
        return d.cpu().numpy()[:, 0]

    def apply_a(z):  # original order in and out, oracle FP64 H-matvec (cluster order inside)
        y = hmul(A, z[perm][:, None])[:, 0]
        out = np.empty_like(y)
        out[perm] = y
        return out

    b = _dev(p.b)
    x = torch.zeros_like(b)
    it, _ = h.solve_gmres(b, x, tol=0.0, restart=30, max_iter=3)
    assert it == 3
    xg = x.cpu().numpy()
    for c in range(p.b.shape[1]):
        xn = _numpy_gmres(apply_a, apply_m, p.b[:, c], 3)
        assert np.max(np.abs(xg[:, c] - xn)) <= 1e-9 * np.max(np.abs(xn)), c
    h.close()


@pytest.mark.parametrize("restart", [30, 2])
def test_gmres_fp32_reaches_1e10(prob, restart):
    """FP32 factors as the preconditioner of FP64 GMRES reach 1e-10 (checked
    with the oracle's H-matvec), with restarts when m = 2, in no more steps than
    iterative refinement needs solves; the solution equals the refined one."""
    import torch
    from paper_1906_00874_gb300 import HLU_FP32
    p = prob
    h = _handle(p, HLU_FP32)
    b = _dev(p.b)
    x = torch.zeros_like(b)
    it, res = h.solve_gmres(b, x, tol=1e-10, restart=restart, max_iter=50)
    assert res <= 1e-10
    xr = torch.zeros_like(b)
    it_ir, res_ir = h.solve_refined(b, xr, tol=1e-10, max_iter=20)
    assert res_ir <= 1e-10 and it <= it_ir
    A = build_hmatrix(p)
    xo = x.cpu().numpy()[p.tree.perm]
    assert np.all(solve_error(A, xo, p.b_perm()) <= 2e-10)
    assert torch.max(torch.abs(x - xr)).item() <= 1e-7 * torch.max(torch.abs(xr)).item()
    h.close()


def test_gmres_fp64_factors_and_states(prob):
    """FP64 factors precondition to a few steps; nrhs = 0 is a no-op; bad restart
    is rejected; a solve before the factorisation is a state error."""
    import torch
    from paper_1906_00874_gb300 import HLU, HLU_FP64
    from paper_1906_00874_gb300.hlu import HLUError
    p = prob
    h = _handle(p, HLU_FP64)
    b = _dev(p.b)
    x = torch.zeros_like(b)
    it, res = h.solve_gmres(b, x, tol=1e-10, restart=30, max_iter=50)
    assert res <= 1e-10 and it <= 4
    assert h.solve_gmres(b[:, :0], x[:, :0]) == (0, 0.0)
    with pytest.raises(HLUError) as e:
        h.solve_gmres(b, x, restart=0)
    assert e.value.status == 1
    h.close()
    h2 = HLU.from_problem(p, precision=HLU_FP64)
    with pytest.raises(HLUError) as e:
        h2.solve_gmres(b, x)
    assert e.value.status == 3
    h2.close()
