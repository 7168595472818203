"""Serving loop on the GPU.  Every request meets its own relative residual of
1e-10 (checked with the oracle's FP64 H-matvec) both alone (its own handle,
factorised and refined) and in the mix; the two solutions then differ by at
most cond(A) times the sum of the two residuals (the bound that those residuals
imply).  Repeats reuse the resident factors; eviction under a small
device-memory budget re-factorises; and the factorisation of a new problem
runs on the device at the same time as the solves of a resident one (CUDA
event timestamps on the two groups' streams)."""
import time

import numpy as np
import pytest

from bem_inputs import build_problem
from oracle import build_hmatrix, densify
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


_COND = {}


def _check(r, p, x_alone):
    A = build_hmatrix(p)
    perm = p.tree.perm
    res_mix = solve_error(A, r.x[perm], r.b[perm])
    res_alone = solve_error(A, x_alone[perm], r.b[perm])
    assert np.all(res_mix <= 1e-10) and np.all(res_alone <= 1e-10)
    if p.n <= 1280:
        key = id(p)
        if key not in _COND:
            _COND[key] = np.linalg.cond(densify(A))
        # x - x' = A^{-1} (r' - r): per column |x - x'| / |x| <= cond(A) (res + res')
        d = np.linalg.norm(r.x - x_alone, axis=0) / np.linalg.norm(x_alone, axis=0)
        assert np.all(d <= _COND[key] * (res_mix + res_alone) * 1.01), (d, _COND[key])


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
    s.drain()
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
        s.drain()
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
        s.drain()
    assert s.stats["evicted_groups"] >= 1 and s.resident_bytes <= budget
    assert reqs[-1].refactored
    for r in reqs:
        _check(r, probs[r.key], _alone(probs[r.key], r.b))
    s.close()


def test_factorisation_overlaps_resident_solves_on_the_device(probs):
    """While a new n = 20480 problem is admitted (planning, then its factorisation on its group's
    stream with half the workers), requests keep arriving for a resident n = 1280 problem and are
    solved on that group's stream: at least one solve starts and ends on the device while the
    factorisation runs (event timestamps on the two streams), and every request, the large one
    included, meets 1e-10."""
    import torch
    from paper_1906_00874_gb300.serve import Request, Server
    big = build_problem(5, 64, 2.0, 1e-4, seed=7, axes=(1.0, 0.8, 0.6))
    s = Server(timeline=True)
    s.submit(Request(0, probs[0], np.ones((probs[0].n, 1)), rid=0))
    s.step(now=0.0)
    s.drain()                                       # problem 0 resident
    ref = torch.cuda.Event(enable_timing=True)
    ref.record()
    torch.cuda.synchronize()
    g = np.random.default_rng(8)
    rb = Request("big", big, g.standard_normal((big.n, 2)), rid=1)
    small = []
    s.submit(rb)
    s.step(now=0.0)
    t0 = time.perf_counter()
    while rb.x is None and time.perf_counter() - t0 < 20.0:  # requests for 0 meanwhile
        r = Request(0, None, g.standard_normal((probs[0].n, 8)), rid=2 + len(small))
        small.append(r)
        s.submit(r)
        s.step(now=0.0)
        time.sleep(0.01)
    s.drain()
    torch.cuda.synchronize()
    assert rb.x is not None and all(r.x is not None for r in small)
    span = {}
    for kind, gid, e0, e1 in s.events:
        span.setdefault(kind, []).append((ref.elapsed_time(e0), ref.elapsed_time(e1), gid))
    big_gid = id(s.where["big"])
    fac = [(a, b) for a, b, gid in span["factor"] if gid == big_gid]
    sol = [(a, b) for a, b, gid in span["solve"] if gid != big_gid]
    assert fac and sol
    assert any(f0 < s0 and s1 < f1 for f0, f1 in fac for s0, s1 in sol), (fac, sol[:5])
    A = build_hmatrix(big)
    assert np.all(solve_error(A, rb.x[big.tree.perm], rb.b[big.tree.perm]) <= 1e-10)
    A0 = build_hmatrix(probs[0])
    for r in small:
        assert np.all(solve_error(A0, r.x[probs[0].tree.perm], r.b[probs[0].tree.perm]) <= 1e-10)
    s.close()
