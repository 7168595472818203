"""Launch settings and plan forms that must not change the factors.

The data-flow graph orders every pair of tasks that touch the same cell, so the factors do not depend on
how many workers run it, on whether product temporaries share device regions (the sharing only adds
order between the earlier and the later user of a region), or on whether a batch was planned as one
forest or problem by problem and joined.  Each case is compared bit for bit with the plain form on the
GPU; the plain form itself is pinned against the oracle in the parity tests."""
import numpy as np
import pytest

from bem_inputs import build_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_1906_00874_gb300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def prob():
    return build_problem(4, 32, 2.0, 1e-4, nrhs=2, axes=(1.0, 0.7, 0.5))


def _factors(h):
    rank, off, data = h.get_factors()
    return rank.copy(), off.copy(), data.copy()


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_worker_count_does_not_change_the_factors(prob, precision):
    """hlu_set_launch: the same handle factorised with every worker, with 100 and with 7 workers
    (hlu_get_launch reports the setting) gives the same factors bit for bit."""
    from paper_1906_00874_gb300 import HLU, HLU_FP32, HLU_FP64
    h = HLU.from_problem(prob, precision=HLU_FP64 if precision == "fp64" else HLU_FP32)
    full = h.get_launch()[0]
    assert full > 100
    h.factor(prob.eps)
    ref = _factors(h)
    for w in (100, 7):
        h.set_launch(w)
        assert h.get_launch() == (w, 0)
        h.factor(prob.eps)
        assert _same(_factors(h), ref), w
    h.set_launch(0)
    assert h.get_launch()[0] == full
    h.close()


def test_shared_temporaries_do_not_change_the_factors_or_the_solve(prob):
    """temp_reuse = 1: a smaller factor arena, the same factors and solution bit for bit."""
    import torch
    from paper_1906_00874_gb300 import HLU, HLU_FP32
    from paper_1906_00874_gb300.hlu import to_device_panel
    out = []
    for reuse in (0, 1):
        h = HLU.from_problem(prob, precision=HLU_FP32, temp_reuse=reuse)
        h.factor(prob.eps)
        b = to_device_panel(prob.b)
        x = torch.zeros_like(b)
        h.solve_refined(b, x, tol=1e-10, max_iter=20)
        out.append((_factors(h), x.cpu().numpy(), h.stats()["device_bytes"]))
        h.close()
    assert _same(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert out[1][2] < out[0][2]


def test_joined_batch_plan_equals_the_forest_plan():
    """A batch planned problem by problem on host threads and joined (the default) and the same batch
    planned as one forest (FLAG_SERIAL_PLAN) give the same factors and solution bit for bit."""
    import torch
    from paper_1906_00874_gb300 import HLU, HLU_FP32
    from paper_1906_00874_gb300.hlu import FLAG_SERIAL_PLAN, to_device_panel
    probs = [build_problem(3, 32, 2.0, 1e-4, nrhs=1),
             build_problem(2, 32, 2.0, 1e-6, nrhs=1, seed=1, axes=(1.0, 0.6, 0.4)),
             build_problem(3, 32, 2.0, 1e-6, nrhs=1, seed=2, axes=(1.0, 0.8, 0.5))]
    b = np.concatenate([p.b for p in probs], axis=0)
    out = []
    for flags in (0, FLAG_SERIAL_PLAN):
        h = HLU.batch(probs, precision=HLU_FP32, flags=flags)
        h.factor([p.eps for p in probs])
        bd = to_device_panel(b)
        x = torch.zeros_like(bd)
        h.solve_refined(bd, x, tol=1e-10, max_iter=20)
        out.append((_factors(h), x.cpu().numpy()))
        h.close()
    assert _same(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
