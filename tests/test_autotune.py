"""The launch-setting tuner (paper_1906_00874_gb300.autotune) on the CPU with a stand-in handle whose
step time depends on its launch settings: the fastest candidate is chosen and applied, and the
choice is cached per structure key and reused without trials."""
import time

from paper_1906_00874_gb300.autotune import candidates, structure_key, tune


class _Handle:
    def __init__(self, cost):
        self.cost = cost
        self.setting = None
        self.calls = 0

    def set_launch(self, workers, flags):
        self.setting = (workers, flags)

    def step(self):
        self.calls += 1
        time.sleep(self.cost[self.setting])


def test_tuner_picks_the_fastest_setting_and_caches_it(tmp_path):
    cands = candidates(4)
    assert len(cands) == 6 and {c["workers"] for c in cands} == {8, 6, 4}
    cost = {(c["workers"], c["flags"]): 0.004 for c in cands}
    cost[(6, 1)] = 0.001
    h = _Handle(cost)
    path = str(tmp_path / "tune.json")
    choice, trials, cached = tune(h, h.step, "k1", cands, reps=2, cache_path=path, sync=lambda: None)
    assert not cached and choice == {"workers": 6, "flags": 1} and h.setting == (6, 1)
    assert len(trials) == 6 and h.calls == 6 * 3  # one warm-up and two timed runs per candidate
    h2 = _Handle(cost)
    choice2, _, cached2 = tune(h2, h2.step, "k1", cands, cache_path=path, sync=lambda: None)
    assert cached2 and choice2 == choice and h2.setting == (6, 1) and h2.calls == 0


def test_structure_key_depends_on_the_structure_and_precision(prob320, prob1280):
    a = structure_key([prob320, prob1280], 1)
    assert a == structure_key([prob320, prob1280], 1)
    assert a != structure_key([prob1280, prob320], 1) and a != structure_key([prob320, prob1280], 0)
