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


def test_pick_reaches_into_nested_entries_and_skips_missing_ones():
    d = {"a": 1, "b": {"c": 2, "d": {"e": 3}}, "x": None}
    assert bench._pick(d, ("a", "b.c", "b.d.e", "b.z", "x", "q")) == {"a": 1, "b.c": 2, "b.d.e": 3, "x": None}


def test_extra_legs_run_as_children_and_report_their_failure(monkeypatch):
    """Each leg is a child process; a child that fails leaves an error entry, and once the wall-time
    budget is spent the remaining legs are skipped without being started."""
    calls = []

    def fake_run(cmd, **kw):
        calls.append(cmd)
        return types.SimpleNamespace(returncode=1, stdout="", stderr="a\nb\nRuntimeError: no device\n")
    monkeypatch.setattr(bench.subprocess, "run", fake_run)
    monkeypatch.setattr(bench, "_T_START", bench.time.time())
    legs = bench.extra_legs(budget_s=1000.0)
    assert set(legs) == {k for k, _, _ in bench.EXTRA_LEGS}
    assert all("no device" in v["error"] for v in legs.values())
    assert len(calls) == len(bench.EXTRA_LEGS) and all("--workload" in c for c in calls)
    calls.clear()
    monkeypatch.setattr(bench, "_T_START", bench.time.time() - 990.0)
    legs = bench.extra_legs(budget_s=1000.0)
    assert not calls and all("skipped" in v for v in legs.values())


def test_extra_legs_keep_the_summary_of_the_childs_line(monkeypatch):
    line = {"value": 40.2, "unit": "problems/s", "config": {"workload": "w"}, "e2e": {"value": 15.0}, "big": [1] * 9}

    def fake_run(cmd, **kw):
        return types.SimpleNamespace(returncode=0, stdout="log line\n" + bench.json.dumps(line) + "\n", stderr="")
    monkeypatch.setattr(bench.subprocess, "run", fake_run)
    monkeypatch.setattr(bench, "_T_START", bench.time.time())
    legs = bench.extra_legs(budget_s=1000.0)
    c4 = legs["c4_ellipsoids64"]
    assert c4["value"] == 40.2 and c4["config.workload"] == "w" and c4["e2e.value"] == 15.0
    assert "big" not in c4 and "wall_s" in c4
