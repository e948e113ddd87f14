"""Failure handling on the GPU without a GPU fault.

A bounded wait on an mbarrier phase that nothing completes gives up, the host reads
KFP_ETIMEOUT, and the same process then sweeps a problem normally: the context is
still usable.  Invalid descriptors are refused on the host before anything launches.
"""
import numpy as np
import pytest

import oracle
from paper_1306_4596_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    from paper_1306_4596_gb300 import swr
    assert swr.kfp_selftest_bounded_wait(1 << 12) == swr.KFP_ETIMEOUT
    assert swr.kfp_selftest_bounded_wait(1 << 16) == swr.KFP_ETIMEOUT
    prob = inputs.small_robin()
    with swr.SWR(prob, "f64") as s:
        s.sweep(3)
        u = s.solution()
    ref = oracle.swr_solve(prob, 3)["u_T"]
    assert np.abs(u - ref).max() <= 1e-12 * np.abs(ref).max()


def test_invalid_limit_is_refused():
    from paper_1306_4596_gb300 import swr
    assert swr.kfp_selftest_bounded_wait(0) == swr.KFP_EINVAL
