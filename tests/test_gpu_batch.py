"""Batched H-LU (hlu_create_batch / hlu_factor_batch): several independent
problems in one handle, factorised and solved in the same launches.

The batch holds diag(A_0, ..., A_{B-1}); blocks that couple two problems are
structurally zero, so every problem's task graph is the one its own handle
plans.  Pinned against single-problem handles (which are pinned against the
oracle elsewhere) and, for the solution, against the oracle's FP64 H-matvec."""
import numpy as np
import pytest

from bem_inputs import build_problem
from oracle import build_hmatrix
from oracle.errors import solve_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_1906_00874_gb300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def probs():
    # different sizes and geometries: sphere, two ellipsoids (ragged n across the batch)
    return [build_problem(3, 32, 2.0, 1e-4, nrhs=2),
            build_problem(2, 32, 2.0, 1e-4, nrhs=2, seed=1, axes=(1.0, 0.6, 0.4)),
            build_problem(3, 32, 2.0, 1e-4, nrhs=2, seed=2, axes=(1.0, 0.8, 0.5))]


def _dev(a):
    from paper_1906_00874_gb300.hlu import to_device_panel
    return to_device_panel(a)


def _stack(probs):
    return np.concatenate([p.b for p in probs], axis=0)


def _single_solutions(probs, eps, precision):
    from paper_1906_00874_gb300 import HLU
    out = []
    for p, e in zip(probs, eps):
        h = HLU.from_problem(p, precision=precision)
        h.factor(e)
        b = _dev(p.b)
        h.solve(b)
        out.append(b.cpu().numpy())
        h.close()
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_solve_equals_single_handles(probs, prec):
    """One factorisation + one solve of the batch gives each problem the
    solution its own handle gives (same tasks, same arithmetic)."""
    from paper_1906_00874_gb300 import HLU, HLU_FP32, HLU_FP64
    precision = HLU_FP64 if prec == "fp64" else HLU_FP32
    h = HLU.batch(probs, precision=precision)
    assert h.count == len(probs) and h.n == sum(p.n for p in probs)
    assert h.sizes == tuple(p.n for p in probs)
    h.factor(1e-4)
    b = _dev(_stack(probs))
    h.solve(b)
    xb = b.cpu().numpy()
    ref = _single_solutions(probs, [1e-4] * len(probs), precision)
    o = 0
    for p, x in zip(probs, ref):
        got = xb[o:o + p.n]
        assert np.max(np.abs(got - x)) <= 1e-12 * np.max(np.abs(x)), (prec, o)
        o += p.n
    h.close()


def test_batch_eps_per_problem(probs):
    """hlu_factor_batch truncates problem i at eps[i]: each block of the
    solution equals the single handle factorised with that eps, and the
    solve error of each problem follows its own tolerance."""
    from paper_1906_00874_gb300 import HLU, HLU_FP64
    eps = [1e-2, 1e-8, 1e-5]
    h = HLU.batch(probs, precision=HLU_FP64)
    h.factor(eps)
    b = _dev(_stack(probs))
    h.solve(b)
    xb = b.cpu().numpy()
    ref = _single_solutions(probs, eps, HLU_FP64)
    o = 0
    errs = []
    for p, x, e in zip(probs, ref, eps):
        got = xb[o:o + p.n]
        assert np.max(np.abs(got - x)) <= 1e-12 * np.max(np.abs(x))
        A = build_hmatrix(p)
        errs.append(np.max(solve_error(A, got[p.tree.perm], p.b_perm())))
        o += p.n
    assert errs[1] < errs[2] < errs[0]
    with pytest.raises(ValueError):
        h.factor([1e-4, 1e-4])
    h.close()


def test_batch_refined_and_gmres_reach_1e10(probs):
    """Iterative refinement and GMRES on the stacked system with FP32 factors
    reach 1e-10 for every problem (oracle FP64 H-matvec per problem), and the
    batch H-matvec is the per-problem H-matvec stacked."""
    import torch
    from paper_1906_00874_gb300 import HLU, HLU_FP32
    h = HLU.batch(probs, precision=HLU_FP32)
    h.factor(1e-4)
    b = _dev(_stack(probs))
    for solver in ("refined", "gmres"):
        x = torch.zeros_like(b)
        if solver == "refined":
            _, res = h.solve_refined(b, x, tol=1e-10, max_iter=20)
        else:
            _, res = h.solve_gmres(b, x, tol=1e-10, restart=30, max_iter=50)
        assert res <= 1e-10, solver
        xh = x.cpu().numpy()
        o = 0
        for p in probs:
            A = build_hmatrix(p)
            assert np.all(solve_error(A, xh[o:o + p.n][p.tree.perm], p.b_perm()) <= 2e-10), (solver, o)
            o += p.n
    y = torch.empty_like(b)
    h.matvec(b, y)
    yb = y.cpu().numpy()
    from oracle.hmatrix import hmul
    o = 0
    for p in probs:
        A = build_hmatrix(p)
        ref = np.empty((p.n, p.b.shape[1]))
        ref[p.tree.perm] = hmul(A, p.b[p.tree.perm])
        assert np.max(np.abs(yb[o:o + p.n] - ref)) <= 1e-12 * np.max(np.abs(ref))
        o += p.n
    h.close()
