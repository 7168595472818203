"""Serving loop for H-LU solves: continuous batching of requests over resident factors.

A request names a problem (an H-matrix, identified by a key) and carries right-hand sides. The server
keeps factorised problems resident on the device in *groups*: one batched handle
(hlu_create_batch) per set of problems that were admitted together. Every step

1. takes all requests that have arrived;
2. admits the problems that are not resident as one new group, factorised in one launch with each
   problem's own eps (hlu_factor_batch); before that, least-recently-used groups are evicted until
   the new group fits the device-memory budget (the handle's own mem_budget check enforces it);
3. solves, per group, all its pending requests in one stacked solve (the block-diagonal system, each
   request's columns in its problem's rows, zeros elsewhere), refined in FP64 to the tolerance for
   every request on its own;
4. returns every request's solution.

Repeated requests for a resident problem therefore cost a solve, not a factorisation. Because the
stacked system is block diagonal, a request's solution does not depend on the other requests in the
step (up to the number of refinement steps the stacked tolerance takes).
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from .hlu import HLU, HLU_FP32, HLUError

ENOMEM = 2


@dataclasses.dataclass
class Request:
    """One solve request: problem `key` (the same key always means the same problem), the problem
    itself (needed only the first time the key is seen, or after eviction), right-hand sides b
    (n x nrhs, original order) and the arrival time (seconds, server clock)."""
    key: object
    problem: object
    b: np.ndarray
    arrival: float = 0.0
    rid: int = 0
    x: np.ndarray | None = None
    done: float | None = None
    refactored: bool = False


class _Group:
    def __init__(self, handle, keys, sizes):
        self.h = handle
        self.keys = list(keys)
        self.offset = dict(zip(keys, np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(int)))
        self.size = dict(zip(keys, sizes))
        self.n = int(sum(sizes))
        self.bytes = handle.stats()["device_bytes"]
        self.last_used = 0


class Server:
    """Continuous-batching H-LU server over resident factors (see the module docstring)."""

    def __init__(self, precision=HLU_FP32, mem_budget=150e9, tol=1e-10, max_iter=30, max_group=64,
                 stream=None, clock=time.perf_counter, device="cuda", handle_type=HLU):
        self.precision = precision
        self.budget = int(mem_budget)
        self.tol = tol
        self.max_iter = max_iter
        self.max_group = max_group
        self.stream = stream
        self.clock = clock
        self.device = device
        self.handle_type = handle_type
        self.groups: list[_Group] = []
        self.where: dict[object, _Group] = {}
        self.queue: collections.deque[Request] = collections.deque()
        self.stats = collections.Counter()
        self._tick = 0

    # ---------------------------------------------------------------- state
    @property
    def resident_bytes(self):
        return sum(g.bytes for g in self.groups)

    def resident(self, key):
        return key in self.where

    def submit(self, req: Request):
        self.queue.append(req)

    def close(self):
        for g in self.groups:
            self._release(g)
        self.groups, self.where = [], {}

    def _release(self, g):
        self.stats["kernels_launched"] += g.h.stats().get("kernels_launched", 0)
        g.h.close()

    def _evict(self, g):
        self.groups.remove(g)
        for k in g.keys:
            del self.where[k]
        self._release(g)
        self.stats["evicted_groups"] += 1

    # ------------------------------------------------------------ admission
    def _admit(self, problems: dict, keep: set):
        """Factorise the new problems as groups of at most max_group, evicting LRU groups (never one
        in `keep`, which this step still solves on) to fit the budget.  A group created here joins
        `keep` at once and is stamped with the current tick, so a later group of the same step never
        evicts it (its requests are still to be solved)."""
        keep = set(keep)
        keys = list(problems)
        while keys:
            part, keys = keys[:self.max_group], keys[self.max_group:]
            while True:
                try:
                    g = self._create(part, problems)
                    break
                except HLUError as e:
                    if e.status != ENOMEM:
                        raise
                    victims = [v for v in self.groups if not (set(v.keys) & keep)]
                    if victims:
                        self._evict(min(victims, key=lambda v: v.last_used))
                    elif len(part) > 1:  # nothing left to evict: admit fewer problems at a time
                        keys = part[len(part) // 2:] + keys
                        part = part[:len(part) // 2]
                    else:
                        raise
            g.last_used = self._tick
            keep.update(g.keys)
            self.groups.append(g)
            for k in g.keys:
                self.where[k] = g

    def _create(self, keys, problems):
        probs = [problems[k] for k in keys]
        budget = self.budget - self.resident_bytes
        if budget <= 0:
            raise HLUError(ENOMEM, "device-memory budget exhausted")
        kw = dict(precision=self.precision, mem_budget=budget, stream=self.stream)
        H = self.handle_type
        h = H.batch(probs, **kw) if len(probs) > 1 else H.from_problem(probs[0], **kw)
        try:
            h.factor([p.eps for p in probs] if len(probs) > 1 else probs[0].eps)
        except Exception:
            h.close()
            raise
        self.stats["factorised_problems"] += len(probs)
        self.stats["groups_created"] += 1
        return _Group(h, keys, [p.n for p in probs])

    # ---------------------------------------------------------------- solve
    def _solve_group(self, g: _Group, reqs):
        import torch

        from .hlu import to_device_panel
        # columns: each problem's requests side by side in its own rows
        col0, width = {}, collections.Counter()
        for r in reqs:
            col0[id(r)] = width[r.key]
            width[r.key] += r.b.shape[1]
        W = max(width.values())
        B = np.zeros((g.n, W), order="F")
        for r in reqs:
            o, c = g.offset[r.key], col0[id(r)]
            B[o:o + g.size[r.key], c:c + r.b.shape[1]] = r.b
        # stacked tolerance: every request's own relative residual ends below self.tol
        colnorm = np.linalg.norm(B, axis=0)
        tol = self.tol
        for r in reqs:
            c = col0[id(r)]
            own = np.linalg.norm(r.b, axis=0)
            ratio = own[own > 0] / colnorm[c:c + r.b.shape[1]][own > 0]
            if ratio.size:
                tol = min(tol, self.tol * float(ratio.min()))
        b = to_device_panel(B, device=self.device)
        x = torch.zeros_like(b)
        it, res = g.h.solve_refined(b, x, tol=tol, max_iter=self.max_iter)
        X = x.cpu().numpy()
        now = self.clock()
        for r in reqs:
            o, c = g.offset[r.key], col0[id(r)]
            r.x = np.array(X[o:o + g.size[r.key], c:c + r.b.shape[1]])
            r.done = now
        self.stats["solves"] += 1
        self.stats["refinement_steps"] += it
        return it, res

    def step(self, now=None):
        """Serve every queued request that has arrived by `now` (default: the clock). Returns them."""
        now = self.clock() if now is None else now
        ready = [r for r in self.queue if r.arrival <= now]
        if not ready:
            return []
        self.queue = collections.deque(r for r in self.queue if r.arrival > now)
        self._tick += 1
        new = {}
        for r in ready:
            if r.key not in self.where and r.key not in new:
                new[r.key] = r.problem
                r.refactored = True
        if new:
            self._admit(new, keep={r.key for r in ready if r.key in self.where})
        by_group = collections.defaultdict(list)
        for r in ready:
            by_group[id(self.where[r.key])].append(r)
        for g in self.groups:
            if id(g) in by_group:
                g.last_used = self._tick
                self._solve_group(g, by_group[id(g)])
        self.stats["requests"] += len(ready)
        return ready
