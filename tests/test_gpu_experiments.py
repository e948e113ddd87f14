"""The experiments of Section 6 on the CUDA path agree with the oracle.

At refinement level j = 0 of Table 1 (hx = hv = dt = 0.01, T = 2, 101 x 201 nodes,
200 steps) the GPU iteration counts to e_mis < 1e-6 in the serial order equal the
oracle's exactly, and a Robin-parameter scan that reuses one solver (factors rebuilt
in place, interface data reset) gives the counts of fresh solvers.
"""
import numpy as np
import pytest

import oracle
from paper_1306_4596_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method,overlap", [("CSWR", 3), ("OSWR(p)", 3), ("OSWR(p,q)", 3), ("OSWR(p)", 0),
                                            ("OSWR(p,q)", 0)])
def test_table1_level0_counts_match_oracle(method, overlap):
    from paper_1306_4596_gb300 import experiments as ex
    robin, p, q = ex.METHODS[method]
    prob = ex._problem(0, overlap, robin, p, q, parallel=False, seed=7)
    gpu = ex.count_iterations(prob)
    ref = oracle.swr_solve(prob, ex.MAX_ITERS, ex.TOL, 1)
    assert gpu["iters"] == ref["iters"], (gpu["iters"], ref["iters"])
    assert gpu["converged"]
    np.testing.assert_allclose(gpu["history"], ref["hist"][:, 0], rtol=1e-9, atol=1e-12)


def test_classical_without_overlap_does_not_converge():
    from paper_1306_4596_gb300 import experiments as ex
    prob = ex._problem(0, 0, False, 1.0, None, parallel=False, seed=7)
    r = ex.count_iterations(prob, 5)
    assert not r["converged"] and r["true_error"] > 1e-2, r


@pytest.mark.parametrize("scheme", [0, 1], ids=["implicit_euler", "split_p1"])
def test_p_scan_reuses_one_solver(scheme):
    from paper_1306_4596_gb300 import experiments as ex
    ps = [3.0, 4.23, 6.0]
    scan = ex.p_scan(ps, j=0, overlap=3, scheme=scheme)
    for p, row in zip(ps, scan):
        fresh = ex.count_iterations(ex._problem(0, 3, True, p, None, parallel=False, seed=7, scheme=scheme))
        assert row["iters"] == fresh["iters"], (p, row, fresh["iters"])
        assert row["converged"]


@pytest.mark.parametrize("method,overlap", [("OSWR(p)", 3), ("OSWR(p,q)", 0)])
def test_table1_level0_split_scheme_matches_oracle(method, overlap):
    from paper_1306_4596_gb300 import experiments as ex
    robin, p, q = ex.METHODS[method]
    prob = ex._problem(0, overlap, robin, p, q, parallel=False, seed=7, scheme=1)
    gpu = ex.count_iterations(prob)
    ref = oracle.swr_solve(prob, ex.MAX_ITERS, ex.TOL, 1)
    assert gpu["iters"] == ref["iters"], (gpu["iters"], ref["iters"])
    np.testing.assert_allclose(gpu["history"], ref["hist"][:, 0], rtol=1e-9, atol=1e-12)
