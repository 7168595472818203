"""Host-side helpers of bench.py (no GPU): the batch split by leaves, the cpu description, and the
configuration record that the native and the reference arm share."""
import types

import bench


class _P:
    def __init__(self, n_leaves, n=0):
        self.n_leaves, self.n = n_leaves, n


def test_balanced_split_keeps_every_problem_once_and_balances_leaves():
    probs = [_P(k) for k in (50, 7, 30, 30, 1, 12, 40, 9)]
    for parts in (1, 2, 3, 4):
        groups = bench._split_balanced(probs, parts)
        flat = sorted(i for g in groups for i in g)
        assert flat == list(range(len(probs)))                 # every problem exactly once
        assert all(g == sorted(g) for g in groups)             # problem order kept inside a group
        loads = [sum(probs[i].n_leaves for i in g) for g in groups]
        assert max(loads) - min(loads) <= max(p.n_leaves for p in probs)


def test_cpu_info_names_the_host():
    info = bench.cpu_info()
    assert info["nproc"] and info["nproc"] >= 1
    assert "cpu_model" in info


def test_native_and_reference_arms_share_the_config():
    args = types.SimpleNamespace(workload="sphere20480", restart=30, solver="ir")
    w = dict(leaf=64, eta=2.0, eps=1e-4)
    p = types.SimpleNamespace(n=20480, n_leaves=14518, nrhs=16, data=types.SimpleNamespace(nbytes=247857288))
    a = bench.workload_config(args, w, p, 1)
    b = bench.workload_config(args, w, p, 1)
    assert a == b and a["n"] == 20480 and a["solver"] == "iterative refinement"
    assert "sphere20480" in a["workload"] and "1e-10" in a["workload"]
