"""Mixed precision (defect correction on the interface problem) against the oracle.

The mixed form runs FP32 strip solves for the corrections and FP64 for the
residual steps, so its converged interface data must match the FP64 fixed point:
the tests iterate the oracle to convergence and require the mixed result to agree
to 1e-10 relative (tolerance of the converged iterate, not of one sweep), with
fewer FP64 iterations than the plain FP64 form needs for the same tolerance.
"""
import numpy as np
import pytest

import oracle
from paper_1306_4596_gb300 import inputs

pytestmark = pytest.mark.gpu


def _swr():
    from paper_1306_4596_gb300 import swr
    return swr


CASES = [
    ("manufactured_robin_p8", lambda: inputs.manufactured(64, 64, 20, 0.1, nstrips=2, overlap=0, robin=True, p=8.0)),
    ("bumps_4_strips_robin", lambda: inputs.gaussian_bumps(96, 128, 30, 2.5e-3, 4, p=6.0, seed=7)),
    ("random_data_dirichlet_ov3", lambda: inputs.random_data(60, 48, 8, 0.01, 3, 3, False, seed=31, nforce=1)),
    ("random_no_bc_robin_pq", lambda: inputs.random_data(90, 256, 6, 0.002, 2, 2, True, p=6.0, q=3.0, seed=32,
                                                         nforce=1, boundary_data=False)),
    # the paper's model problem: periodic x and zero flux in v, with this library's scheme
    # in the serial order, and with the split P1 scheme of Section 6.2
    ("model_problem_serial_order", lambda: inputs.gaussian_bumps(96, 128, 30, 2.5e-3, 4, p=6.0, seed=7).replace(
        neumann_v=True, periodic_x=True, gauss_seidel=True)),
    ("model_problem_split_scheme", lambda: inputs.gaussian_bumps(96, 128, 30, 2.5e-3, 4, p=6.0, seed=7).replace(
        neumann_v=True, periodic_x=True, scheme=1)),
]


@pytest.mark.parametrize("label,factory", CASES, ids=[c[0] for c in CASES])
def test_mixed_converges_to_the_fp64_fixed_point(label, factory):
    swr = _swr()
    prob = factory()
    ref = oracle.swr_solve(prob, 2000, 1e-14, 0)
    with swr.SWR(prob, "mixed") as s:
        n = s.sweep(20, 1e-12, 1)
        u = s.solution()
        lam = s.traces()
        hist = s.error()[3]
        cnt = s.counters()
    assert hist[-1, 0] < 1e-12, hist
    scale_u = np.abs(ref["u_T"]).max()
    assert np.abs(u - ref["u_T"]).max() <= 1e-10 * scale_u
    # the mixed form returns lambda (its last FP64 step measured it); the oracle's
    # fixed point agrees to the convergence tolerance
    scale_l = np.abs(ref["lam"]).max()
    assert np.abs(lam - ref["lam"]).max() <= 1e-9 * scale_l
    assert cnt["fp64_iterations"] == n and n <= 6, cnt
    assert cnt["fp32_iterations"] > 0


def test_mixed_uses_fewer_fp64_iterations_than_fp64():
    swr = _swr()
    prob = inputs.gaussian_bumps(96, 128, 30, 2.5e-3, 4, p=6.0, seed=7)
    with swr.SWR(prob, "f64") as s:
        n64 = s.sweep(400, 1e-11, 1)
        e64 = s.error()[0]
    with swr.SWR(prob, "mixed") as s:
        nm = s.sweep(20, 1e-11, 1)
        em = s.error()[0]
    assert e64 < 1e-11 and em < 1e-11
    assert nm < n64 / 3, (nm, n64)


def test_mixed_single_strip_is_fp64():
    swr = _swr()
    prob = inputs.random_data(70, 32, 5, 0.01, 1, 0, False, seed=10, nforce=1)
    with swr.SWR(prob, "mixed") as s:
        s.sweep(1)
        u = s.solution()
    np.testing.assert_allclose(u, oracle.monolithic(prob), rtol=0, atol=1e-12 * np.abs(u).max())
