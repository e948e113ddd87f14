"""The CUDA path against the oracle on the workloads the benchmark reports beyond the
headline one.

* Adjoint workload, full size (512 x 1024 cells, 8 Robin strips, 7 interface
  parameters, nt = 500, K = 10): the gradient of the interface mismatch from the
  GPU's discrete adjoint against the oracle's adjoint of the same K iterations.
* Mixed-precision workload (4096 x 8192 cells, 16 Robin strips, nt = 4000) scaled
  down by 32 in x, v and t (128 x 256 cells, nt = 125, the same box, strips, Robin
  parameter, CFL 0.8192 and T = 0.2), small enough for the oracle to reach its
  fixed point (e_chg < 1e-13, 152 iterations): the FP64 and the mixed-precision GPU
  results, each iterated to convergence, against that fixed point element by
  element.  The error of each result is printed with -s.
"""
import numpy as np
import pytest

import oracle
from paper_1306_4596_gb300 import inputs

pytestmark = pytest.mark.gpu


def _swr():
    from paper_1306_4596_gb300 import swr
    return swr


def test_adjoint_workload_gradient_matches_oracle_adjoint():
    swr = _swr()
    prob = inputs.adjoint_workload()
    K = 10
    J_o, gp_o, gq_o = oracle.swr_adjoint(prob, K)
    with swr.SWR(prob) as s:
        J, gp, gq = s.gradient(K)
    scale = max(np.abs(gp_o).max(), np.abs(gq_o).max())
    err_J = abs(J - J_o) / J_o
    err_g = max(np.abs(gp - gp_o).max(), np.abs(gq - gq_o).max()) / scale
    print(f"adjoint workload: J rel err {err_J:.2e}, gradient rel err {err_g:.2e}")
    assert err_J <= 1e-11
    assert err_g <= 1e-10, (gp, gp_o, gq, gq_o)


def reduced_mixed_workload():
    """The mixed-precision workload with every grid size divided by 32."""
    full = inputs.mixed_precision_workload()
    return inputs.gaussian_bumps(full.nx // 32, full.nv // 32, full.nt // 32, full.dt * 32, nstrips=16, p=4.0,
                                 seed=4)


@pytest.fixture(scope="module")
def reduced_fixed_point():
    prob = reduced_mixed_workload()
    ref = oracle.swr_solve(prob, 3000, 1e-13, 0)
    assert ref["hist"][-1, 1] < 1e-13
    return prob, ref


def test_reduced_mixed_workload_fp64_matches_oracle_fixed_point(reduced_fixed_point):
    swr = _swr()
    prob, ref = reduced_fixed_point
    with swr.SWR(prob, "f64") as s:
        n = s.sweep(3000, 1e-13, 0)
        u, lam = s.solution(), s.traces()
    assert n == ref["iters"]
    err_u = np.abs(u - ref["u_T"]).max() / np.abs(ref["u_T"]).max()
    err_l = np.abs(lam - ref["lam"]).max() / np.abs(ref["lam"]).max()
    print(f"reduced mixed workload, FP64 GPU ({n} iterations): solution rel err {err_u:.2e}, "
          f"interface data rel err {err_l:.2e}")
    assert err_u <= 1e-12 and err_l <= 1e-12


def test_reduced_mixed_workload_mixed_matches_oracle_fixed_point(reduced_fixed_point):
    swr = _swr()
    prob, ref = reduced_fixed_point
    with swr.SWR(prob, "mixed") as s:
        n = s.sweep(20, 1e-12, 1)
        u, lam = s.solution(), s.traces()
        hist = s.error()[3]
        cnt = s.counters()
    assert hist[-1, 0] < 1e-12
    err_u = np.abs(u - ref["u_T"]).max() / np.abs(ref["u_T"]).max()
    err_l = np.abs(lam - ref["lam"]).max() / np.abs(ref["lam"]).max()
    print(f"reduced mixed workload, mixed precision ({cnt['fp64_iterations']} FP64 + "
          f"{cnt['fp32_iterations']} FP32 iterations): solution rel err {err_u:.2e}, "
          f"interface data rel err {err_l:.2e}")
    assert err_u <= 1e-10 and err_l <= 1e-9
    assert n <= 6
