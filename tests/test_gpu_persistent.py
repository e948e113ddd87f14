"""The streamed sweep (the interior passes of an iteration in one co-resident
launch, units waiting on their column neighbours' completion counters) against the
one-launch-per-pass sweep and the oracle.

Both forms run the same pass code on the same data in the same order per column, so
their results must agree bit for bit; the parity with the oracle is then that of
the per-pass form (tests/test_gpu_parity.py runs every parity case on the default,
per-pass, form).  The stall check runs the bounded-wait failure path of
the counters on purpose: one unit never reports completion, its neighbours give up
after a short limit and every block leaves; the next sweep of the same handle must
be unaffected.
"""
import numpy as np
import pytest

import oracle
from paper_1306_4596_gb300 import inputs

pytestmark = pytest.mark.gpu

RD = inputs.random_data


def _run(prob, iters, precision="f64", **kw):
    from paper_1306_4596_gb300 import swr
    with swr.SWR(prob, precision, **kw) as s:
        s.sweep(iters)
        return {"u_T": s.solution(), "lam": s.traces(), "bands": s.bands(), "hist": s.error()[3],
                "stats": s.stats()}


def _same(a, b):
    for key in ("u_T", "lam", "bands", "hist"):
        assert np.array_equal(a[key], b[key]), key


CASES = [
    ("small_robin", inputs.small_robin, 3),
    ("small_dirichlet", inputs.small_dirichlet, 3),
    ("two_passes_only", lambda: RD(40, 16, 2, 0.01, 2, 2, True, seed=80, nforce=1), 2),
    ("three_passes", lambda: RD(61, 32, 3, 0.01, 4, 0, True, p=3.0, q=1.5, seed=81, nforce=1), 2),
    ("fast_robin_time_forcing", lambda: RD(77, 192, 7, 0.002, 3, 0, True, p=4.0, q=2.0, seed=82, nforce=1,
                                           boundary_data=False), 2),
    ("fast_const_forcing_ov4", lambda: RD(250, 300, 6, 0.002, 3, 4, True, p=5.0, seed=83, nforce=1,
                                          constant_in_time=True, boundary_data=False), 2),
    ("no_forcing_dirichlet", lambda: RD(150, 128, 5, 0.003, 2, 4, False, seed=84, nforce=0), 2),
    ("bumps_8_strips", lambda: inputs.gaussian_bumps(300, 512, 40, 8e-4, 8, p=4.0, seed=85), 2),
]


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("label,factory,iters", CASES, ids=[c[0] for c in CASES])
def test_persistent_equals_per_pass(label, factory, iters, precision):
    prob = factory()
    a = _run(prob, iters, precision, persistent=True)
    b = _run(prob, iters, precision, persistent=False)
    _same(a, b)
    if prob.nt > 1:  # first pass, interior passes in one launch, last pass (+ exchange, error)
        assert a["stats"]["launches_per_iter"] == 5
        assert b["stats"]["launches_per_iter"] == prob.nt + 3


def test_persistent_serial_order_matches_oracle():
    prob = RD(90, 256, 6, 0.002, 4, 2, True, p=5.0, seed=86, nforce=1, boundary_data=False).replace(
        gauss_seidel=True)
    a = _run(prob, 3, persistent=True)
    _same(a, _run(prob, 3, persistent=False))
    lam = prob.lam0.copy()
    for _ in range(3):
        lam, bands, u_T = oracle.swr_iteration(prob, lam)
    assert np.abs(a["u_T"] - u_T).max() <= 1e-12 * np.abs(u_T).max()
    assert np.abs(a["lam"] - lam).max() <= 1e-12 * np.abs(lam).max()


def test_more_units_than_resident_blocks():
    """The 4096 x 8192, 16-strip grid (560 units, several per block) on a short window:
    blocks walk several units per pass; bitwise equal to the per-pass form, and the
    first iteration agrees with the oracle on sampled columns."""
    prob = inputs.mixed_precision_workload().replace(nt=6)
    prob.f_time = prob.f_time[:, :7].copy()
    a = _run(prob, 1)  # chosen by default: 560 units per pass, more than resident blocks
    assert a["stats"]["launches_per_iter"] == 5
    b = _run(prob, 1, persistent=False)
    _same(a, b)
    lam, bands, u_T = oracle.swr_iteration(prob, None)
    assert np.abs(a["u_T"] - u_T).max() <= 1e-12 * np.abs(u_T).max()
    assert np.abs(a["lam"] - lam).max() <= 1e-12 * np.abs(lam).max()


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_stalled_unit_times_out_and_handle_recovers(precision):
    from paper_1306_4596_gb300 import swr
    prob = inputs.gaussian_bumps(300, 512, 40, 8e-4, 8, p=4.0, seed=87)
    ref = _run(prob, 2, precision)
    with swr.SWR(prob, precision, persistent=True) as s:
        s.sweep(1)
        # unit 3 (strip 1, first column block) never reports; its neighbours give up after 50 ms
        st = swr.kfp_swr_selftest_stall(s.h, 3, 0.05)
        assert st == swr.KFP_ETIMEOUT, swr.STATUS_NAMES.get(st, st)
        assert swr.kfp_swr_selftest_stall(s.h, 10 ** 6, 0.05) == swr.KFP_EINVAL
        s.sweep(1)
        assert np.array_equal(s.solution(), ref["u_T"])
        assert np.array_equal(s.traces(), ref["lam"])
        assert np.array_equal(s.error()[3], ref["hist"])


def test_stall_check_needs_the_persistent_sweep():
    from paper_1306_4596_gb300 import swr
    with swr.SWR(inputs.small_robin()) as s:
        assert swr.kfp_swr_selftest_stall(s.h, 0, 0.05) == swr.KFP_ENOTSUP


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("label,factory,iters", [CASES[4], CASES[5], CASES[7]], ids=[CASES[4][0], CASES[5][0],
                                                                                    CASES[7][0]])
def test_tile_shapes_are_bitwise_identical(label, factory, iters, precision):
    """Every tile shape (16- or 8-row ring stages, one or two blocks per SM), in the
    per-pass and in the streamed form, gives the same bits."""
    prob = factory()
    ref = _run(prob, iters, precision, persistent=False, tile_shape=0)
    for shape in (0, 1, 2):
        for persistent in (False, True):
            if (shape, persistent) != (0, False):
                _same(ref, _run(prob, iters, precision, persistent=persistent, tile_shape=shape))
