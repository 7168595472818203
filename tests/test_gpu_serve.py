"""Serving loop on the GPU: every request's solution is the one the problem
gets alone (its own handle, factorised and refined to 1e-10), whatever else
is in the step; repeats reuse the resident factors; eviction under a small
device-memory budget re-factorises and still gives the same solutions.  The
residuals are checked with the oracle's FP64 H-matvec."""
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
    return {0: build_problem(3, 32, 2.0, 1e-4, seed=0),
            1: build_problem(2, 32, 2.0, 1e-6, seed=1, axes=(1.0, 0.7, 0.5)),
            2: build_problem(3, 32, 2.0, 1e-4, seed=2, axes=(1.0, 0.9, 0.6)),
            3: build_problem(2, 32, 2.0, 1e-4, seed=3, axes=(1.0, 0.5, 0.5))}


def _alone(p, b):
    import torch
    from paper_1906_00874_gb300 import HLU, HLU_FP32
    from paper_1906_00874_gb300.hlu import to_device_panel
    h = HLU.from_problem(p, precision=HLU_FP32)
    h.factor(p.eps)
    bd = to_device_panel(b)
    x = torch.zeros_like(bd)
    h.solve_refined(bd, x, tol=1e-10, max_iter=30)
    h.close()
    return x.cpu().numpy()


def _check(r, p, x_alone):
    A = build_hmatrix(p)
    perm = p.tree.perm
    assert np.all(solve_error(A, r.x[perm], r.b[perm]) <= 1.5e-10)
    assert np.max(np.abs(r.x - x_alone)) <= 1e-8 * np.max(np.abs(x_alone))


def _stream(probs, seed=5):
    from paper_1906_00874_gb300.serve import Request
    g = np.random.default_rng(seed)
    keys = [0, 1, 0, 2, 3, 1, 2, 0]  # repeats
    out = []
    for i, k in enumerate(keys):
        nrhs = int(g.integers(1, 5))
        out.append(Request(k, probs[k], g.standard_normal((probs[k].n, nrhs)), arrival=float(i // 3), rid=i))
    return out


def test_mixed_steps_equal_alone_and_reuse_factors(probs):
    from paper_1906_00874_gb300.serve import Server
    reqs = _stream(probs)
    s = Server()
    for r in reqs:
        s.submit(r)
    for t in range(3):
        s.step(now=float(t))
    assert all(r.x is not None for r in reqs)
    assert s.stats["factorised_problems"] == 4  # every problem factorised once
    assert [r.refactored for r in reqs] == [True, True, False, True, True, False, False, False]
    for r in reqs:
        _check(r, probs[r.key], _alone(probs[r.key], r.b))
    s.close()


def test_small_budget_evicts_and_refactorises(probs):
    from paper_1906_00874_gb300.serve import Request, Server
    size = {}
    for k in (0, 1, 2):
        s = Server()
        s.submit(Request(k, probs[k], np.ones((probs[k].n, 1))))
        s.step(now=0.0)
        size[k] = s.resident_bytes
        s.close()
    # room for either n = 1280 problem plus the n = 320 one, never for both n = 1280 problems
    budget = max(size[0], size[2]) + size[1] + 1
    assert budget < size[0] + size[2]
    s = Server(mem_budget=budget)
    g = np.random.default_rng(3)
    order = [0, 2, 0, 1, 2]
    reqs = [Request(k, probs[k], g.standard_normal((probs[k].n, 2)), arrival=float(i), rid=i)
            for i, k in enumerate(order)]
    for r in reqs:
        s.submit(r)
        s.step(now=r.arrival)
    assert s.stats["evicted_groups"] >= 1 and s.resident_bytes <= budget
    assert reqs[-1].refactored
    for r in reqs:
        _check(r, probs[r.key], _alone(probs[r.key], r.b))
    s.close()
