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
    # the inverses are extra factorisation tasks; the factorisation itself is unchanged
    assert on["factor_tasks"] > off["factor_tasks"] and on["matvec_tasks"] == off["matvec_tasks"]


@pytest.mark.parametrize("inv_block", [-1, 0])
def test_batch_plans_only_its_problems_tasks(inv_block):
    from paper_1906_00874_gb300.hlu import plan_info
    probs = [build_problem(3, 32, 2.0, 1e-4), build_problem(2, 32, 2.0, 1e-4, seed=1, axes=(1.0, 0.6, 0.4)),
             build_problem(2, 32, 2.0, 1e-4, seed=2, axes=(1.0, 0.8, 0.5))]
    one = [plan_info(p, inv_block=inv_block) for p in probs]
    batch = plan_info(probs, inv_block=inv_block)
    for key in ("factor_tasks", "factor_edges", "solve_tasks", "matvec_tasks", "inverse_blocks"):
        assert batch[key] == sum(o[key] for o in one), key
    for key in ("factor_levels", "solve_levels"):
        assert batch[key] == max(o[key] for o in one), key
