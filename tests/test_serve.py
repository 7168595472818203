"""Host logic of the serving loop (paper_1906_00874_gb300.serve) on the CPU:
request packing into the stacked block-diagonal system, the stacked
tolerance, admission under the device-memory budget and LRU eviction, and the
threads that run admissions and solves while step() returns at once.

The handle is a dense stand-in with the library's interface (no GPU): each
problem is a small dense matrix, the stacked solve is an exact dense solve
of the block-diagonal system, and creation fails with the library's ENOMEM
status when it would exceed the handle's memory budget."""
import time

import numpy as np
import pytest

from paper_1906_00874_gb300.hlu import HLUError
from paper_1906_00874_gb300.serve import Request, Server


class _Prob:
    def __init__(self, n, seed, eps=1e-4):
        g = np.random.default_rng(seed)
        self.n, self.eps = n, eps
        self.A = g.standard_normal((n, n)) + n * np.eye(n)


class _FakeHLU:
    created = []

    def __init__(self, probs, mem_budget):
        self.probs = probs
        self.bytes = sum(8 * p.n * p.n for p in probs)
        if mem_budget and self.bytes > mem_budget:
            raise HLUError(2, "fake: over budget")
        self.factored = None
        self.solve_tols = []
        _FakeHLU.created.append(self)

    @classmethod
    def batch(cls, probs, precision=None, mem_budget=0, stream=None):
        return cls(list(probs), mem_budget)

    @classmethod
    def from_problem(cls, p, precision=None, mem_budget=0, stream=None):
        return cls([p], mem_budget)

    def stats(self):
        return {"device_bytes": self.bytes}

    def factor(self, eps):
        self.factored = list(np.atleast_1d(eps))

    def solve_refined(self, b, x, tol=1e-10, max_iter=20):
        import scipy.linalg
        self.solve_tols.append(tol)
        A = scipy.linalg.block_diag(*[p.A for p in self.probs])
        import torch
        x.copy_(torch.from_numpy(np.linalg.solve(A, b.numpy())))
        return 1, 0.0

    def close(self):
        self.closed = True


def _server(budget=1e9, **kw):
    _FakeHLU.created = []
    return Server(mem_budget=budget, device="cpu", handle_type=_FakeHLU, **kw)


def _step(s, now):
    """Dispatch what has arrived by `now` and wait for the jobs: the requests completed meanwhile."""
    out = s.step(now=now)
    return out + s.drain()


def test_packing_repeats_and_per_problem_eps():
    probs = {k: _Prob(n, k, eps=10.0 ** -(3 + k)) for k, n in enumerate((5, 7, 4))}
    g = np.random.default_rng(9)
    reqs = [Request(k, probs[k], g.standard_normal((probs[k].n, c)), rid=i)
            for i, (k, c) in enumerate([(0, 2), (1, 1), (0, 3), (2, 2), (1, 1)])]
    s = _server()
    for r in reqs:
        s.submit(r)
    out = _step(s, 0.0)
    assert len(out) == 5 and len(_FakeHLU.created) == 1
    h = _FakeHLU.created[0]
    assert h.factored == [probs[k].eps for k in (0, 1, 2)]  # one group, one eps per problem
    for r in reqs:
        assert np.allclose(probs[r.key].A @ r.x, r.b, atol=1e-10)
    # the stacked tolerance bounds every request's own relative residual
    assert h.solve_tols[-1] <= 1e-10
    # repeats of resident problems are solved, not factorised again
    r2 = Request(1, None, g.standard_normal((7, 4)), rid=9)
    s.submit(r2)
    _step(s, 1.0)
    assert len(_FakeHLU.created) == 1 and s.stats["factorised_problems"] == 3
    assert np.allclose(probs[1].A @ r2.x, r2.b, atol=1e-10)


def test_only_arrived_requests_are_served():
    p = _Prob(3, 0)
    s = _server()
    s.submit(Request("a", p, np.ones((3, 1)), arrival=5.0))
    assert _step(s, 1.0) == []
    assert len(_step(s, 5.0)) == 1


def test_budget_evicts_least_recently_used_group():
    probs = {k: _Prob(10, k) for k in range(3)}   # 800 bytes each
    s = _server(budget=1700)                      # room for two problems
    for t, k in enumerate([0, 1, 0, 2]):          # 1 is the least recently used when 2 arrives
        s.submit(Request(k, probs[k], np.ones((10, 1)), arrival=float(t), rid=t))
        _step(s, float(t))
    assert s.resident(0) and s.resident(2) and not s.resident(1)
    assert s.stats["evicted_groups"] == 1 and s.resident_bytes <= 1700
    r = Request(1, probs[1], np.ones((10, 1)), arrival=9.0, rid=9)
    s.submit(r)
    _step(s, 9.0)
    assert r.refactored and np.allclose(probs[1].A @ r.x, r.b)


def test_group_too_large_is_split_and_hopeless_problem_raises():
    probs = {k: _Prob(10, k) for k in range(4)}
    s = _server(budget=1700)
    for k in range(2):
        s.submit(Request(k, probs[k], np.ones((10, 1)), rid=k))
    _step(s, 0.0)
    assert s.resident(0) and s.resident(1)
    big = _Prob(20, 7)                            # 3200 bytes: over the budget on its own
    s.submit(Request("big", big, np.ones((20, 1)), rid=5))
    with pytest.raises(HLUError):
        _step(s, 1.0)


def test_new_problems_are_grouped_by_max_group():
    """Problems arriving together are admitted as groups of at most max_group problems; each group
    is one handle, factorised once, and every request is answered from its own problem's rows."""
    probs = {k: _Prob(4 + k, k) for k in range(5)}
    s = _server(max_group=2)
    g = np.random.default_rng(1)
    reqs = [Request(k, probs[k], g.standard_normal((probs[k].n, 1)), rid=k) for k in range(5)]
    for r in reqs:
        s.submit(r)
    out = _step(s, 0.0)
    assert len(out) == 5 and len(_FakeHLU.created) == 3
    assert sorted(len(h.probs) for h in _FakeHLU.created) == [1, 2, 2]
    assert s.stats["groups_created"] == 3 and s.stats["solves"] == 3
    for r in reqs:
        assert np.allclose(probs[r.key].A @ r.x, r.b, atol=1e-10)


def test_groups_admitted_in_one_step_are_not_evicted_by_later_groups():
    """Three new problems admitted one group each (max_group=1) under a budget for three problems, with
    one idle old group resident: the old group is the one evicted, never a group created earlier in
    the same step, and every request is answered."""
    probs = {k: _Prob(10, k) for k in range(4)}   # 800 bytes each
    s = _server(budget=2500, max_group=1)         # room for three problems
    s.submit(Request("old", probs[3], np.ones((10, 1)), rid=0))
    _step(s, 0.0)
    assert s.resident("old")
    g = np.random.default_rng(3)
    reqs = [Request(k, probs[k], g.standard_normal((10, 1)), arrival=1.0, rid=1 + k) for k in range(3)]
    for r in reqs:
        s.submit(r)
    out = _step(s, 1.0)
    assert len(out) == 3
    assert not s.resident("old") and all(s.resident(k) for k in range(3))
    assert s.stats["evicted_groups"] == 1
    for r in reqs:
        assert np.allclose(probs[r.key].A @ r.x, r.b, atol=1e-10)


def test_halved_group_admits_its_second_half_by_evicting_the_first():
    """Two new problems that do not fit together (one at a time does): the group is halved, the
    first half is solved as soon as it is factorised, then evicted to make room for the second
    half, and both requests are answered."""
    probs = {k: _Prob(10, k) for k in range(2)}   # 800 bytes each
    s = _server(budget=1000, max_group=2)
    g = np.random.default_rng(5)
    reqs = [Request(k, probs[k], g.standard_normal((10, 1)), rid=k) for k in range(2)]
    for r in reqs:
        s.submit(r)
    out = _step(s, 0.0)
    assert sorted(r.rid for r in out) == [0, 1]
    assert s.stats["groups_created"] == 2 and s.stats["evicted_groups"] == 1
    for r in reqs:
        assert np.allclose(probs[r.key].A @ r.x, r.b, atol=1e-10)


class _SlowHLU(_FakeHLU):
    """A stand-in whose factorisation and solves take time (sleep, as a device call would block the
    calling thread without holding the interpreter lock)."""
    factor_s = 0.2
    solve_s = 0.2
    spans = []

    def factor(self, eps):
        t0 = time.perf_counter()
        time.sleep(self.factor_s)
        _SlowHLU.spans.append(("factor", t0, time.perf_counter()))
        super().factor(eps)

    def solve_refined(self, b, x, tol=1e-10, max_iter=20):
        t0 = time.perf_counter()
        time.sleep(self.solve_s)
        out = super().solve_refined(b, x, tol, max_iter)
        _SlowHLU.spans.append(("solve", t0, time.perf_counter()))
        return out


def test_admission_and_solves_run_concurrently_and_step_does_not_block():
    """A request for a resident problem is solved while a new problem is being factorised (the two
    run on different threads at the same time), step() returns without waiting for either, and a
    request that arrives for a problem under admission is solved once its group exists."""
    _SlowHLU.spans = []
    probs = {k: _Prob(6, k) for k in range(3)}
    s = Server(mem_budget=1e9, device="cpu", handle_type=_SlowHLU)
    s.submit(Request(0, probs[0], np.ones((6, 1)), rid=0))
    _step(s, 0.0)                                 # problem 0 resident
    _SlowHLU.spans = []
    g = np.random.default_rng(4)
    reqs = [Request(1, probs[1], g.standard_normal((6, 1)), arrival=1.0, rid=1),
            Request(0, None, g.standard_normal((6, 2)), arrival=1.0, rid=2),
            Request(1, None, g.standard_normal((6, 1)), arrival=2.0, rid=3)]
    for r in reqs:
        s.submit(r)
    t0 = time.perf_counter()
    first = s.step(now=1.0)
    assert time.perf_counter() - t0 < 0.1 and first == []   # dispatch only
    second = s.step(now=2.0)                     # problem 1 is still being admitted
    out = first + second + s.drain()
    assert sorted(r.rid for r in out) == [1, 2, 3]
    for r in reqs:
        assert np.allclose(probs[r.key].A @ r.x, r.b, atol=1e-10)
    fac = [sp for sp in _SlowHLU.spans if sp[0] == "factor"]
    sol = [sp for sp in _SlowHLU.spans if sp[0] == "solve"]
    assert len(fac) == 1 and len(sol) == 2
    # the solve of the resident problem 0 overlaps the factorisation of problem 1
    assert any(a[1] < b[2] and b[1] < a[2] for a in fac for b in sol)
    s.close()


def test_problems_arriving_while_admission_is_busy_are_admitted_together():
    """With one admission thread busy on a first problem, three problems that arrive meanwhile wait
    in the queue and are admitted by the next job as one group (one handle), and every request is
    answered from its own problem's rows."""
    _SlowHLU.spans = []
    _FakeHLU.created = []
    probs = {k: _Prob(5 + k, k) for k in range(4)}
    s = Server(mem_budget=1e9, device="cpu", handle_type=_SlowHLU, admit_threads=1)
    g = np.random.default_rng(6)
    reqs = [Request(k, probs[k], g.standard_normal((probs[k].n, 1)), arrival=float(k > 0), rid=k) for k in range(4)]
    for r in reqs:
        s.submit(r)
    out = s.step(now=0.0)          # problem 0: its admission starts (factorisation takes 0.2 s)
    time.sleep(0.05)
    out += s.step(now=1.0)         # problems 1-3 arrive while the only admission thread is busy
    out += s.drain()
    assert sorted(r.rid for r in out) == [0, 1, 2, 3]
    assert sorted(len(h.probs) for h in _FakeHLU.created) == [1, 3]
    assert s.stats["groups_created"] == 2
    for r in reqs:
        assert np.allclose(probs[r.key].A @ r.x, r.b, atol=1e-10)
    s.close()


def test_a_group_takes_more_problems_only_within_its_unknowns_cap():
    """Queued problems are grouped in arrival order while the group's unknowns stay within
    max_group_n: two small problems form one group, the large one that follows its own."""
    _SlowHLU.spans = []
    _FakeHLU.created = []
    probs = {0: _Prob(5, 0), 1: _Prob(5, 1), 2: _Prob(6, 2), 3: _Prob(30, 3)}
    s = Server(mem_budget=1e9, device="cpu", handle_type=_SlowHLU, admit_threads=1, max_group_n=20)
    g = np.random.default_rng(7)
    reqs = [Request(k, probs[k], g.standard_normal((probs[k].n, 1)), arrival=float(k > 0), rid=k) for k in range(4)]
    for r in reqs:
        s.submit(r)
    out = s.step(now=0.0)          # problem 0 alone keeps the only admission thread busy
    time.sleep(0.05)
    out += s.step(now=1.0)         # 1 and 2 (11 unknowns) are grouped; 3 (30) would pass the cap
    out += s.drain()
    assert sorted(r.rid for r in out) == [0, 1, 2, 3]
    assert [sorted(p.n for p in h.probs) for h in _FakeHLU.created] == [[5], [5, 6], [30]]
    for r in reqs:
        assert np.allclose(probs[r.key].A @ r.x, r.b, atol=1e-10)
    s.close()


def test_memory_estimate_first_then_the_free_budget():
    """A creation first reserves its estimated memory (leaves x bytes_per_leaf + a margin), at most the
    free budget: with a budget that one reservation fills, a second new problem waits for the first
    creation and is then admitted with what is left; both requests are answered."""
    probs = {k: _Prob(10, k) for k in range(2)}   # 800 bytes each
    for p in probs.values():
        p.n_leaves = 4
    s = _server(budget=2000, max_group=1, admit_threads=2)
    g = np.random.default_rng(9)
    reqs = [Request(k, probs[k], g.standard_normal((10, 1)), rid=k) for k in range(2)]
    for r in reqs:
        s.submit(r)
    out = _step(s, 0.0)
    assert sorted(r.rid for r in out) == [0, 1]
    assert s.stats["groups_created"] == 2 and s.stats.get("evicted_groups", 0) == 0
    for r in reqs:
        assert np.allclose(probs[r.key].A @ r.x, r.b, atol=1e-10)
