"""Launch-setting tuner for H-LU handles: chooses, from timed trials, how many worker CTAs the
data-flow launches of a handle use and whether its dense products run on the tensor cores.

The task graph is fixed by the H-matrix structure; what remains free at run time is the shape of the
persistent launch that executes it (hlu_set_launch): the number of resident workers (all, or fewer so
that fewer tasks compete for the SMs' FP64 units, shared memory bandwidth and L2) and the product
path of the FP32 factorisation (CUDA cores or tcgen05 tensor cores).  tune() times `step` (for example
factorise and solve) under every candidate on the given handle, keeps the fastest, and caches the
choice per structure key in a JSON file, so that later handles with the same structure take it
without trials.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

from .hlu import FLAG_TENSOR


def structure_key(problems, precision):
    """A key of the H-matrix structure of a list of problems (sizes, leaf sizes, tolerances, leaf
    counts and kinds) and the precision: the inputs the task graph and its cost depend on."""
    h = hashlib.sha1()
    h.update(str(int(precision)).encode())
    for p in problems:
        h.update(f"{p.n}:{getattr(p, 'leaf', 0)}:{p.eps:g}:{p.n_leaves}:{int((p.kind == 1).sum())};".encode())
    return h.hexdigest()[:20]


def default_cache():
    d = os.environ.get("HLU_CACHE_DIR") or os.path.join(os.path.expanduser("~"), ".cache", "hlu_gb300")
    os.makedirs(d, exist_ok=True)
    return os.path.join(d, "launch_tuning.json")


def candidates(sms, tensor=True):
    """Worker counts (two per SM, one and a half, one) times the product path."""
    out = []
    for w in (2 * sms, (3 * sms) // 2, sms):
        for f in ((0, FLAG_TENSOR) if tensor else (0,)):
            out.append({"workers": int(w), "flags": int(f)})
    return out


def _time(step, reps, sync):
    best = float("inf")
    for _ in range(reps):
        sync()
        t0 = time.perf_counter()
        step()
        sync()
        best = min(best, time.perf_counter() - t0)
    return best


def tune(handle, step, key, cands, reps=2, cache_path=None, sync=None, use_cache=True):
    """Best launch setting for `handle` among `cands` ({"workers", "flags"} dicts) by the shortest
    time of `step()` (the best of `reps` runs after one warm-up); the choice is applied to the handle
    and stored under `key`.  Returns (choice, trials: [(setting, seconds)], from_cache)."""
    if sync is None:
        import torch
        sync = torch.cuda.synchronize
    cache_path = cache_path or default_cache()
    cache = {}
    if use_cache and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        c = cache[key]["choice"]
        handle.set_launch(c["workers"], c["flags"])
        return c, cache[key]["trials"], True
    trials = []
    for c in cands:
        handle.set_launch(c["workers"], c["flags"])
        step()  # warm-up under this setting
        trials.append((c, _time(step, reps, sync)))
    choice = min(trials, key=lambda t: t[1])[0]
    handle.set_launch(choice["workers"], choice["flags"])
    cache[key] = {"choice": choice, "trials": [[c, s] for c, s in trials]}
    tmp = f"{cache_path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, cache_path)
    return choice, trials, False
