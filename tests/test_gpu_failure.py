"""Failure detection without a GPU fault: a task that never becomes ready
(host-side injection through hlu_inject_stall) makes the data-flow kernel's
bounded waits run out; the call returns HLU_ETIMEOUT, the kernel ends, and the
same handle factorises correctly afterwards."""
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


def test_stalled_task_times_out_and_the_handle_recovers():
    import time

    from paper_1906_00874_gb300 import HLU, HLU_FP64
    from paper_1906_00874_gb300.hlu import HLUError
    p = build_problem(3, 32, 2.0, 1e-4, nrhs=1)
    h = HLU.from_problem(p, precision=HLU_FP64, timeout_s=0.5)
    h.inject_stall()
    t0 = time.perf_counter()
    with pytest.raises(HLUError) as e:
        h.factor(p.eps)
    assert e.value.status == 6  # HLU_ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    # the injection is consumed; the device and the handle are usable again
    h.factor(p.eps)
    ref = HLU.from_problem(p, precision=HLU_FP64)
    ref.factor(p.eps)
    r1, o1, d1 = h.get_factors()
    r2, o2, d2 = ref.get_factors()
    assert np.array_equal(r1, r2) and np.array_equal(d1, d2)
    h.close()
    ref.close()
