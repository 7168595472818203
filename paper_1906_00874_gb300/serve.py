"""Serving loop for H-LU solves: continuous batching of requests over resident factors.

A request names a problem (an H-matrix, identified by a key) and carries right-hand sides. The server
keeps factorised problems resident on the device in *groups*: one batched handle (hlu_create_batch)
per set of problems that were admitted together, each group with its own CUDA stream.

Work runs on host threads that drive the library (its calls release the Python interpreter lock), so
that the device holds several requests' work at once:

* admission threads create and factorise new groups (each problem with its own eps,
  hlu_factor_batch), several at once so that their host planning runs in parallel; the creations in
  flight share the budget left free (each asks for an estimate of its group's memory first).  New
  problems wait in one queue, and a free thread takes the oldest as one group: up to max_group of
  them while the group's unknowns stay within max_group_n, so problems that arrive while every
  admission thread is busy are admitted together without small ones waiting for many large ones.
  An admission evicts least-recently-used idle groups when the device-memory budget is short; when
  nothing can be evicted yet it waits until a running job ends and frees memory, and it splits a
  group that cannot fit on its own;
* solve threads run, per group, one stacked refined solve of the requests that have arrived for it
  (the block-diagonal system, each request's columns in its problem's rows, zeros elsewhere, FP64
  refinement to the tolerance for every request on its own).  A group runs one job at a time, in
  order: its solves start once its factorisation is done.

Every data-flow launch of a group uses at most `workers` worker CTAs (half of the resident slots by
default), so a group's factorisation and another group's solve share the GPU instead of queueing
behind each other. step() only dispatches and collects: requests that arrive while others are on the
GPU are admitted at once, as slots and memory free up. Because the stacked system is block diagonal, a
request's solution depends on the other requests of its solve only through the number of refinement
steps, and every request meets its own residual tolerance.
"""
from __future__ import annotations

import collections
import concurrent.futures
import dataclasses
import threading
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
    refactored: bool = False   # this request's problem was (re)factorised for it
    waited: bool = False       # it waited for the admission of its problem
    resident_at: float | None = None  # server clock: its group resident (or the arrival if it was)
    solve_at: float | None = None     # server clock: its stacked solve started
    iters: int = 0


class _Group:
    def __init__(self, handle, keys, sizes, stream):
        self.h = handle
        self.keys = list(keys)
        self.offset = dict(zip(keys, np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(int)))
        self.size = dict(zip(keys, sizes))
        self.n = int(sum(sizes))
        self.bytes = handle.stats()["device_bytes"]
        self.stream = stream
        self.last_used = 0
        self.busy = 0          # jobs queued or running on the group
        self.tail = None       # future of its last job (jobs of a group run in order)


class Server:
    """Continuous-batching H-LU server over resident factors (see the module docstring)."""

    def __init__(self, precision=HLU_FP32, mem_budget=150e9, tol=1e-10, max_iter=30, max_group=16,
                 stream=None, clock=time.perf_counter, device="cuda", handle_type=HLU, workers=None,
                 solve_threads=2, admit_threads=8, stream_factory=None, timeline=False, temp_reuse=0,
                 max_group_n=65536, bytes_per_leaf=400e3):
        self.precision = precision
        self.budget = int(mem_budget)
        self.tol = tol
        self.max_iter = max_iter
        self.max_group = max_group
        self.max_group_n = max_group_n      # a group takes more problems only while its unknowns stay below
        self.bytes_per_leaf = bytes_per_leaf  # device-memory estimate of a new group, per leaf
        self.clock = clock
        self.device = device
        self.handle_type = handle_type
        self.workers = self._default_workers() if workers is None else int(workers)
        self.stream_factory = stream_factory or self._default_stream_factory(stream)
        self.timeline = timeline
        self.temp_reuse = temp_reuse  # hlu_opts.temp_reuse of the groups (1: half the memory, slower planning)
        self.groups: list[_Group] = []
        self.where: dict[object, _Group] = {}
        self.admitting: set = set()  # keys dispatched for admission and not resident yet
        self.waiting: dict[object, list] = collections.defaultdict(list)  # key being admitted -> requests
        self.queue: collections.deque[Request] = collections.deque()
        self.stats = collections.Counter()
        self.events = []           # (kind, group id, start event, end event) when timeline is on
        self.admissions = []       # per created group: problems, unknowns, create s, factorise s
        self._tick = 0
        self._lock = threading.RLock()
        self._freed = threading.Condition(self._lock)
        self._done: list[Request] = []
        self._errors: list[BaseException] = []
        self._creating = 0         # creations in flight (they share the free budget)
        self._reserved = 0         # bytes of budget handed to the creations in flight
        self._pending = collections.deque()  # keys dispatched, not yet taken by an admission job
        self._pending_probs: dict = {}
        self._admit_futs: list = []
        self.admit_threads = int(admit_threads)
        self._admit_pool = concurrent.futures.ThreadPoolExecutor(admit_threads, thread_name_prefix="hlu-admit")
        self._solve_pool = concurrent.futures.ThreadPoolExecutor(solve_threads, thread_name_prefix="hlu-solve")

    def _default_workers(self):
        if self.device != "cuda":
            return 0
        import torch
        return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count

    def _default_stream_factory(self, stream):
        if self.device != "cuda":
            return lambda: None
        import torch
        if stream is not None:  # one given stream for every group: no device overlap between groups
            given = stream if isinstance(stream, torch.cuda.Stream) else torch.cuda.ExternalStream(int(stream))
            return lambda: given
        return torch.cuda.Stream

    # ---------------------------------------------------------------- state
    @property
    def resident_bytes(self):
        return sum(g.bytes for g in self.groups)

    def resident(self, key):
        return key in self.where

    def submit(self, req: Request):
        self.queue.append(req)

    def close(self):
        self.drain()
        self._admit_pool.shutdown(wait=True)
        self._solve_pool.shutdown(wait=True)
        for g in self.groups:
            self._release(g)
        self.groups, self.where = [], {}

    def drain(self):
        """Wait until every dispatched job has finished; returns the requests completed since the
        last step() or drain()."""
        while True:
            with self._lock:
                self._admit_futs = [f for f in self._admit_futs if not f.done()]
                futs = list(self._admit_futs) + [g.tail for g in self.groups if g.tail is not None]
            pending = [f for f in futs if not f.done()]
            if not pending:
                break
            concurrent.futures.wait(pending)
        return self._collect()

    def _release(self, g):
        self.stats["kernels_launched"] += g.h.stats().get("kernels_launched", 0)
        g.h.close()

    def _evict(self, g):
        self.groups.remove(g)
        for k in g.keys:
            del self.where[k]
        self._release(g)
        self.stats["evicted_groups"] += 1

    def _stream_ptr(self, s):
        if s is None:
            return None
        return getattr(s, "cuda_stream", s)

    def _record(self, s):
        if not self.timeline or s is None or self.device != "cuda" or not hasattr(s, "record_event"):
            return None
        import torch
        e = torch.cuda.Event(enable_timing=True)
        e.record(s)
        return e

    # ------------------------------------------------------------ admission
    def _admit_next(self):
        """Admission thread: take the oldest dispatched problems that no job has taken yet as one
        group (the requests that arrived while every admission thread was busy are admitted
        together: at most max_group problems, and more than one only while the group's unknowns
        stay within max_group_n, so that a small problem does not wait for a long factorisation of
        many large ones) and admit them; repeat while problems are queued."""
        while True:
            with self._lock:
                part, total = [], 0
                while self._pending and len(part) < self.max_group:
                    nk = getattr(self._pending_probs[self._pending[0]], "n", 0)
                    if part and total + nk > self.max_group_n:
                        break
                    part.append(self._pending.popleft())
                    total += nk
                problems = {k: self._pending_probs.pop(k) for k in part}
            if not part:
                return
            try:
                self._admit_job(part, problems)
            except BaseException:
                with self._lock:  # forget the keys it did not admit; their waiting requests are dropped
                    for k in part:
                        if k not in self.where:
                            self.admitting.discard(k)
                            self.waiting.pop(k, None)
                raise

    def _admit_job(self, keys, problems):
        """Create and factorise the groups of `keys` (at most max_group problems each), evicting idle
        LRU groups to fit the budget, waiting for memory while other creations or solves are
        running, and halving a group that cannot fit by itself.  Each group is registered (and the
        solves of its waiting requests queued) as soon as it is factorised."""
        keys = list(keys)
        while keys:
            part, keys = keys[:self.max_group], keys[self.max_group:]
            exclusive = False
            while True:
                try:
                    self._create(part, problems, exclusive)
                    break
                except HLUError as e:
                    if e.status != ENOMEM:
                        raise
                    with self._lock:
                        if not exclusive:  # a share was not enough: next, all the free budget
                            exclusive = True
                            continue
                        if self._creating > 0:  # another creation holds part of the budget
                            self._freed.wait(timeout=1.0)
                            continue
                        idle = [v for v in self.groups if v.busy == 0]
                        if idle:
                            self._evict(min(idle, key=lambda v: v.last_used))
                            continue
                        if any(v.busy for v in self.groups):  # memory frees when a solve ends
                            self._freed.wait(timeout=1.0)
                            continue
                    if len(part) > 1:  # nothing to evict and nothing running: fewer at a time
                        keys = part[len(part) // 2:] + keys
                        part = part[:len(part) // 2]
                    else:
                        raise

    def _register(self, g):
        """Make a new group resident and queue the solves of the requests waiting for its keys
        (called with the lock held)."""
        self.groups.append(g)
        g.last_used = self._tick
        reqs = []
        for k in g.keys:
            self.where[k] = g
            self.admitting.discard(k)
            reqs += self.waiting.pop(k, [])
        now = self.clock()
        for r in reqs:
            r.resident_at = now
        if reqs:
            self._chain_solve(g, reqs)

    def _create(self, keys, problems, exclusive=False):
        """Create, factorise and register one group.  Creations run on several admission threads at
        once (the host planning of one problem does not wait for another's).  The budget left free
        by the resident groups and the creations in flight is split equally over the admissions
        that still need a share (at most one per admission thread); an exclusive creation (a retry
        after a share was too small) waits until no other creation is in flight and takes all of
        it.  The group's registration and the release of its share happen under one lock, so that a
        waiting admission never sees memory as neither reserved nor resident."""
        probs = [problems[k] for k in keys]
        est = None
        if self.bytes_per_leaf and all(hasattr(p, "n_leaves") for p in probs):
            est = int(self.bytes_per_leaf * sum(p.n_leaves for p in probs)) + (64 << 20)
        with self._lock:
            if exclusive:
                while self._creating > 0:
                    self._freed.wait(timeout=1.0)
                claim = 1
            else:
                # this creation, those in flight, and the groups still to be taken from the queue
                waiting_groups = -(-len(self._pending) // self.max_group)
                claim = max(1, min(self.admit_threads, self._creating + 1 + waiting_groups) - self._creating)
            free = self.budget - self.resident_bytes - self._reserved
            # the estimate of the group's memory when there is one (a first try; a group that needs
            # more comes back exclusive), else an equal share of the free budget
            budget = min(free, est) if est is not None and not exclusive else free // claim
            if budget <= 0:
                raise HLUError(ENOMEM, "device-memory budget exhausted")
            self._creating += 1
            self._reserved += budget
        g = None
        try:
            g = self._create_in(keys, probs, budget)
            return g
        finally:
            with self._lock:
                self._creating -= 1
                self._reserved -= budget
                if g is not None:
                    self._register(g)
                self._freed.notify_all()

    def _create_in(self, keys, probs, budget):
        stream = self.stream_factory()
        kw = dict(precision=self.precision, mem_budget=budget, stream=self._stream_ptr(stream))
        if self.temp_reuse:
            kw["temp_reuse"] = self.temp_reuse
        if self.workers:
            kw["workers"] = self.workers
        H = self.handle_type
        t0 = self.clock()
        h = H.batch(probs, **kw) if len(probs) > 1 else H.from_problem(probs[0], **kw)
        t1 = self.clock()
        e0 = self._record(stream)  # the factorisation's device work only (after the host planning)
        try:
            h.factor([p.eps for p in probs] if len(probs) > 1 else probs[0].eps)
        except Exception:
            h.close()
            raise
        e1 = self._record(stream)
        t2 = self.clock()
        g = _Group(h, keys, [p.n for p in probs], stream)
        with self._lock:
            self.stats["factorised_problems"] += len(probs)
            self.stats["groups_created"] += 1
            # (problems, unknowns, seconds to create the handle, seconds to factorise)
            self.admissions.append((len(probs), g.n, t1 - t0, t2 - t1))
            if e0 is not None:
                self.events.append(("factor", id(g), e0, e1))
        return g

    # ---------------------------------------------------------------- solve
    def _solve_job(self, g: _Group, reqs):
        """Solve thread: one stacked refined solve of `reqs` on group g (its own stream)."""
        try:
            if self.device == "cuda":
                import torch
                with torch.cuda.stream(g.stream):
                    self._solve_group(g, reqs)
            else:
                self._solve_group(g, reqs)
        finally:
            with self._lock:
                g.busy -= 1
                self._freed.notify_all()

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
        t_solve = self.clock()
        for r in reqs:
            r.solve_at = t_solve
        e0 = self._record(g.stream)
        b = to_device_panel(B, device=self.device)  # a host-to-device copy, no kernel
        x = torch.empty_like(b)  # written by the refinement (which starts from zero itself)
        it, res = g.h.solve_refined(b, x, tol=tol, max_iter=self.max_iter)
        X = x.cpu().numpy()
        e1 = self._record(g.stream)
        now = self.clock()
        for r in reqs:
            o, c = g.offset[r.key], col0[id(r)]
            r.x = np.array(X[o:o + g.size[r.key], c:c + r.b.shape[1]])
            r.iters = it
            r.done = now
        with self._lock:
            self.stats["solves"] += 1
            self.stats["refinement_steps"] += it
            if e0 is not None:
                self.events.append(("solve", id(g), e0, e1))
            self._done.extend(reqs)

    # --------------------------------------------------------------- driver
    def _on_error(self, fut):
        e = fut.exception()
        if e is not None:
            with self._lock:
                self._errors.append(e)

    def _chain_solve(self, g: _Group, reqs, after=None):
        """Queue a solve of reqs on g after the group's previous job (and `after`, a future)."""
        prev = [f for f in (g.tail, after) if f is not None]

        def run():
            for f in prev:
                f.result()
            self._solve_job(g, reqs)
        g.busy += 1
        g.last_used = self._tick
        g.tail = self._solve_pool.submit(run)
        g.tail.add_done_callback(self._on_error)

    def _collect(self):
        with self._lock:
            if self._errors:
                e = self._errors.pop(0)
                raise e
            out, self._done = self._done, []
        self.stats["requests"] += len(out)
        return out

    def step(self, now=None):
        """Dispatch every queued request that has arrived by `now` (default: the clock) and return
        the requests whose solutions are ready since the last call (without waiting)."""
        now = self.clock() if now is None else now
        ready = [r for r in self.queue if r.arrival <= now]
        if ready:
            self.queue = collections.deque(r for r in self.queue if r.arrival > now)
            with self._lock:
                self._tick += 1
                by_group = collections.defaultdict(list)
                new = {}
                for r in ready:
                    if r.key in self.where:
                        by_group[id(self.where[r.key])].append(r)
                        r.resident_at = now
                    else:  # solved once its group is registered (_register)
                        if r.key not in self.admitting and r.key not in new:
                            new[r.key] = r.problem
                            r.refactored = True
                        self.waiting[r.key].append(r)
                        r.waited = True
                for g in self.groups:
                    if id(g) in by_group:
                        self._chain_solve(g, by_group[id(g)])
                keys = list(new)
                self._pending += keys
                self._pending_probs.update(new)
                self.admitting.update(keys)
                for _ in range(-(-len(keys) // self.max_group)):  # one job per group of new keys
                    fut = self._admit_pool.submit(self._admit_next)
                    fut.add_done_callback(self._on_error)
                    self._admit_futs.append(fut)
        return self._collect()

    def serve(self, requests, poll=1e-4):
        """Submit `requests` (their arrival times on the server clock) and serve them until every
        one has its solution; returns them in completion order."""
        for r in requests:
            self.submit(r)
        out = []
        while len(out) < len(requests):
            now = self.clock()
            out += self.step(now)
            if len(out) >= len(requests):
                break
            nxt = min((r.arrival for r in self.queue), default=None)
            wait = poll if nxt is None else max(0.0, min(poll, nxt - now))
            time.sleep(wait)
        return out
