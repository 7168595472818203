"""Parity at the benchmark's full size: the n = 20480 unit sphere (leaf 64,
eta = 2, eps = 1e-4, 16 right-hand sides), in the launch configuration the
benchmark times (one handle, whole task graph, refinement to 1e-10).

The oracle factorises the same problem on the host (about a minute); the
tolerance rules are those of test_gpu_parity: rounding-level agreement when
every truncation rank agrees, otherwise at most a few rank flips and agreement
within 10 eps.  The FP32 arm is checked by the property that holds at any size:
FP64 refinement reaches ||b - A_H x|| <= 1e-10 ||b||, with the residual
recomputed by the oracle's own H-matvec.
"""
import numpy as np
import pytest

from bem_inputs import WORKLOADS, build_problem
from oracle import HLUOracle, build_hmatrix, densify
from oracle.errors import lu_solve, solve_error
from oracle.hmatrix import hmul

from gpu_helpers import factors_as_problem, gpu_factor, rank_agreement

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    from paper_1906_00874_gb300 import build
    build.build()
    p = build_problem(**WORKLOADS["sphere20480"])
    o = HLUOracle(p, p.eps).factor()
    return p, o


def _leafwise_max_diff(q, o, amax):
    G = {l.leaf_id: l for l in build_hmatrix(q).leaves()}
    worst = 0.0
    for l in o.A.leaves():
        worst = max(worst, float(np.max(np.abs(densify(G[l.leaf_id]) - densify(l)))) if l.m and l.n else 0.0)
    return worst / amax


def test_fullsize_fp64_factor_parity(big):
    p, o = big
    h = gpu_factor(p)
    q = factors_as_problem(p, h)
    same, tot = rank_agreement(o, q)
    amax = max(float(np.max(np.abs(p.data))), 1e-300)
    err = _leafwise_max_diff(q, o, amax)
    if same == tot:
        assert err <= 1e-10, err
    else:
        assert tot - same <= max(2, tot // 500), (same, tot)
        assert err <= 10 * p.eps, err
    # the solve with the same factors
    from paper_1906_00874_gb300.hlu import to_device_panel
    b = to_device_panel(p.b)
    h.solve(b)
    xo = lu_solve(o.A, p.b_perm())
    x = b.cpu().numpy()[p.tree.perm]
    assert np.max(np.abs(x - xo)) / np.max(np.abs(xo)) <= (1e-10 if same == tot else 10 * p.eps)
    h.close()


def test_fullsize_fp32_refinement_reaches_1e10(big):
    import torch
    from paper_1906_00874_gb300 import HLU_FP32
    from paper_1906_00874_gb300.hlu import to_device_panel
    p, _ = big
    h = gpu_factor(p, precision=HLU_FP32)
    b = to_device_panel(p.b)
    x = torch.zeros_like(b)
    iters, res = h.solve_refined(b, x, tol=1e-10, max_iter=30)
    assert res <= 1e-10 and iters <= 8
    A = build_hmatrix(p)
    xr = x.cpu().numpy()[p.tree.perm]
    assert np.all(solve_error(A, xr, p.b_perm()) <= 2e-10)
    h.close()


def test_fullsize_matvec_matches_oracle(big):
    import torch
    from paper_1906_00874_gb300 import HLU
    from paper_1906_00874_gb300.hlu import to_device_panel
    p, _ = big
    h = HLU.from_problem(p)
    xs = np.random.default_rng(5).standard_normal((p.n, 3))
    y = to_device_panel(np.zeros_like(xs))
    h.matvec(to_device_panel(xs), y)
    yo = np.empty_like(xs)
    yo[p.tree.perm] = hmul(build_hmatrix(p), xs[p.tree.perm])
    assert np.max(np.abs(y.cpu().numpy() - yo)) / np.max(np.abs(yo)) <= 1e-13
    torch.cuda.synchronize()
    h.close()
