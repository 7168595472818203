"""The two execution schedules of the task graph give the same factors.

The data-flow schedule (one persistent launch, a task starts when its own
predecessors are done) and the wave schedule (one launch per dependency level)
run the same tasks on the same inputs; no task combines partial results
through atomics, so if the dependency edges are complete the factors are
bitwise identical.  A missing edge would show up here as a data race.
"""
import numpy as np
import pytest

from bem_inputs import build_problem

from gpu_helpers import gpu_factor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1906_00874_gb300 import build
    build.build()


@pytest.mark.parametrize("precision", [0, 1])
def test_dataflow_equals_waves(precision):
    from paper_1906_00874_gb300.hlu import SCHED_DATAFLOW, SCHED_WAVES
    p = build_problem(4, 32, 2.0, 1e-4, nrhs=1)
    h1 = gpu_factor(p, precision=precision, schedule=SCHED_DATAFLOW)
    h2 = gpu_factor(p, precision=precision, schedule=SCHED_WAVES)
    r1, o1, d1 = h1.get_factors()
    r2, o2, d2 = h2.get_factors()
    assert np.array_equal(r1, r2)
    assert np.array_equal(d1, d2)
    for _ in range(2):  # repeated data-flow runs are identical too
        h1.factor(p.eps)
        assert np.array_equal(h1.get_factors()[2], d1)
    h1.close()
    h2.close()
