"""Host planning without a device (hlu_plan_info_get / hlu_plan_info_batch):
the inverse-block solve shortens the solve's dependency chain; a batch plans
exactly its problems' own tasks (no task couples two problems)."""
import pytest

from bem_inputs import build_problem


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1906_00874_gb300 import build, hlu
    build.build()
    return hlu.load()


def test_inverse_blocks_shorten_the_solve(prob1280):
    from paper_1906_00874_gb300.hlu import plan_info
    off = plan_info(prob1280, inv_block=-1)
    on = plan_info(prob1280)
    small = plan_info(prob1280, inv_block=64)
    assert off["inverse_blocks"] == 0 and on["inverse_blocks"] >= 2 and small["inverse_blocks"] > on["inverse_blocks"]
    assert on["solve_levels"] < small["solve_levels"] < off["solve_levels"]
    assert on["solve_critical_us"] < off["solve_critical_us"]
    assert 0.0 < off["factor_critical_us"] <= on["factor_critical_us"]
    # the inverses are extra factorisation tasks; the factorisation itself is unchanged
    assert on["factor_tasks"] > off["factor_tasks"] and on["matvec_tasks"] == off["matvec_tasks"]


@pytest.mark.parametrize("serial", [False, True])
@pytest.mark.parametrize("inv_block", [-1, 0])
def test_batch_plans_only_its_problems_tasks(inv_block, serial):
    """A batch plans each problem's tasks and dependencies and nothing else, whether the problems
    are planned on their own threads and joined (default) or as one forest (FLAG_SERIAL_PLAN)."""
    from paper_1906_00874_gb300.hlu import FLAG_SERIAL_PLAN, plan_info
    probs = [build_problem(3, 32, 2.0, 1e-4), build_problem(2, 32, 2.0, 1e-4, seed=1, axes=(1.0, 0.6, 0.4)),
             build_problem(2, 32, 2.0, 1e-4, seed=2, axes=(1.0, 0.8, 0.5))]
    one = [plan_info(p, inv_block=inv_block) for p in probs]
    batch = plan_info(probs, inv_block=inv_block, flags=FLAG_SERIAL_PLAN if serial else 0)
    for key in ("factor_tasks", "factor_edges", "solve_tasks", "matvec_tasks", "inverse_blocks"):
        assert batch[key] == sum(o[key] for o in one), key
    for key in ("factor_levels", "solve_levels"):
        assert batch[key] == max(o[key] for o in one), key
    assert batch["factor_critical_us"] == pytest.approx(max(o["factor_critical_us"] for o in one))


def test_wave_order_does_not_change_the_graph(prob1280):
    """The wave schedule sorts each kind's tasks by wave; the data-flow schedule keeps emission order.
    Both plan the same graph; only the wave schedule lays out rounded-addition scratch in the arena
    (the data-flow workers have their own)."""
    from paper_1906_00874_gb300.hlu import SCHED_WAVES, plan_info
    a = plan_info(prob1280)
    b = plan_info(prob1280, schedule=SCHED_WAVES)
    for key in ("factor_tasks", "factor_edges", "factor_levels", "solve_tasks", "solve_levels", "matvec_tasks",
                "inverse_blocks"):
        assert a[key] == b[key], key
    assert a["factor_elems"] < b["factor_elems"]


@pytest.mark.parametrize("case", [dict(r=3, leaf=32, eta=0.5, eps=1e-4, dim=1),
                                  dict(r=3, leaf=32, eta=1.0, eps=1e-4, dim=2),
                                  dict(r=3, leaf=32, eta=0.0, eps=1e-4)])
def test_variants_plan(case):
    """The d = 1, 2 problems and the dense-only structure (eta = 0: every leaf dense) plan on the
    host, with inverse blocks for the solve."""
    from paper_1906_00874_gb300.hlu import plan_info
    p = build_problem(nrhs=1, **case)
    info = plan_info(p)
    assert info["factor_tasks"] > 0 and info["inverse_blocks"] >= 1
    if case["eta"] == 0.0:
        assert (p.kind == 0).all()


def test_temporaries_sharing_regions_keep_the_levels_and_shrink_the_arena(prob1280):
    """temp_reuse: product temporaries whose dependency-level intervals do not overlap share regions.
    The graph keeps its number of levels (the added orderings go from a lower level to a higher
    one), the factor arena shrinks, and the temporaries' level peak bounds what they need."""
    from paper_1906_00874_gb300.hlu import plan_info
    off = plan_info(prob1280)
    on = plan_info(prob1280, temp_reuse=1)
    assert on["factor_levels"] == off["factor_levels"] and on["factor_tasks"] == off["factor_tasks"]
    assert on["factor_edges"] >= off["factor_edges"]
    assert on["factor_elems"] < off["factor_elems"]
    saved = off["factor_elems"] - on["factor_elems"]
    assert 0 < off["factor_temp_peak_elems"] <= off["factor_temp_elems"]
    assert saved <= off["factor_temp_elems"] - off["factor_temp_peak_elems"]
