"""Batched sweep: many uneven problems swept together (first pass, streamed interior
passes, last pass per iteration).

Every problem of a batch runs exactly the arithmetic of its own handle, so its
results must be bit-identical to a single-problem run, for every launch shape the
autotuner can pick, and within the FP64 parity tolerance of the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1306_4596_gb300 import inputs

pytestmark = pytest.mark.gpu

RD = inputs.random_data


def batch_problems():
    return [
        inputs.small_robin(),                                                           # time-dependent forcing
        RD(90, 256, 6, 0.002, 2, 3, False, seed=40, nforce=1, boundary_data=False),     # Dirichlet, overlap 3
        RD(77, 192, 4, 0.002, 3, 0, True, p=4.0, q=2.0, seed=41, nforce=0, boundary_data=False),  # no forcing
        RD(150, 300, 7, 0.002, 3, 4, True, p=5.0, seed=42, nforce=1, constant_in_time=True,
           boundary_data=False),                                                        # pre-scaled forcing
        RD(37, 24, 3, 0.01, 3, 2, False, seed=43, nforce=1),                            # boundary data
        inputs.gaussian_bumps(200, 256, 12, 1e-3, 4, p=6.0, seed=44),
        RD(29, 16, 1, 0.02, 2, 1, True, p=2.0, seed=45, nforce=1),                      # a single step
    ]


def single_results(prob, precision, iters):
    from paper_1306_4596_gb300 import swr
    with swr.SWR(prob, precision) as s:
        s.sweep(iters)
        return s.solution(), s.traces(), s.error()[3]


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_batch_equals_single_problem_runs(precision):
    from paper_1306_4596_gb300 import swr
    probs = batch_problems()
    iters = 3
    ref = [single_results(p, precision, iters) for p in probs]
    for bps, order, shape in ((0, 0, 1), (1, 0, 0), (1, 1, 2), (2, 1, 1), (0, 1, 0)):
        with swr.Batch(probs, precision) as b:
            b.configure(bps, order, shape)
            n = b.sweep(iters)
            assert n == iters
            for i, p in enumerate(probs):
                v = b.view(i)
                u, lam, hist = v.solution(), v.traces(), v.error()[3]
                assert np.array_equal(u, ref[i][0]), (bps, order, shape, i)
                assert np.array_equal(lam, ref[i][1]), (bps, order, shape, i)
                assert np.array_equal(hist, ref[i][2]), (bps, order, shape, i)


# strip heights - 1 (nv / S) whose chunk count equals the ring depth of each tile
# shape: shape 0 has 16-row stages (4 FP64 / 8 FP32 of them), shape 1 8-row stages
# (4 / 8), shape 2 8-row stages (6 / 12)
RING_ROWS = {(0, "f64"): 60, (0, "f32"): 120, (1, "f64"): 30, (1, "f32"): 60, (2, "f64"): 46, (2, "f32"): 94}


@pytest.mark.parametrize("shape", [0, 1, 2])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_batch_units_as_long_as_the_ring(precision, shape):
    """Problems whose strips take exactly as many chunks as the ring has stages, so
    that a unit's successor starts in the stage of the unit's own first chunk while
    that unit is still running, with different problems (other arrays) back to back."""
    from paper_1306_4596_gb300 import swr
    rows = RING_ROWS[(shape, precision)]
    probs = [RD(90 + 7 * i, rows * S, 5 + i, 0.002, S, 0, True, p=3.0 + i, seed=90 + i, nforce=1,
                boundary_data=False) for i, S in enumerate((2, 3, 4, 2, 3))]
    ref = [single_results(p, precision, 2) for p in probs]
    with swr.Batch(probs, precision) as b:
        b.configure(0, 1, shape)
        b.sweep(2)
        for i in range(len(probs)):
            v = b.view(i)
            assert np.array_equal(v.solution(), ref[i][0]), i
            assert np.array_equal(v.traces(), ref[i][1]), i


def test_batch_matches_oracle():
    from paper_1306_4596_gb300 import swr
    probs = batch_problems()
    with swr.Batch(probs, "f64") as b:
        b.sweep(2)
        for i, p in enumerate(probs):
            lam = p.lam0.copy() if p.lam0 is not None else np.zeros(oracle.trace_shape(p))
            for _ in range(2):
                lam, bands, u_T = oracle.swr_iteration(p, lam)
            v = b.view(i)
            assert np.abs(v.solution() - u_T).max() <= 1e-12 * np.abs(u_T).max()
            if p.nstrips > 1:
                assert np.abs(v.traces() - lam).max() <= 1e-12 * np.abs(lam).max()


def test_batch_tolerance_and_autotune(tmp_path, monkeypatch):
    from paper_1306_4596_gb300 import autotune, swr
    monkeypatch.setenv("KFP_SWR_CACHE", str(tmp_path))
    probs = [inputs.manufactured(64, 64, 20, 0.1, nstrips=2, overlap=0, robin=True, p=8.0),
             inputs.gaussian_bumps(96, 128, 30, 2.5e-3, 4, p=6.0, seed=7)]
    with swr.Batch(probs, "f64") as b:
        t1 = autotune.tune(b, "f64")
        assert not t1["cached"] and len(t1["candidates"]) == len(autotune.CANDIDATES) >= 8
        n = b.sweep(300, 1e-12, 1)
        assert n < 300
        for i in range(2):
            assert b.view(i).error()[0] < 1e-12
    with swr.Batch(probs, "f64") as b:
        t2 = autotune.tune(b, "f64")
        assert t2["cached"] and (t2["blocks_per_sm"], t2["unit_order"], t2["tile_shape"]) == (
            t1["blocks_per_sm"], t1["unit_order"], t1["tile_shape"])


def test_batch_rejects_unsupported():
    from paper_1306_4596_gb300 import swr
    with pytest.raises(swr.KfpError) as ei:
        swr.Batch([inputs.small_robin()], "mixed")
    assert ei.value.status == swr.KFP_ENOTSUP
    with pytest.raises(swr.KfpError) as ei:
        swr.Batch([RD(61, 32, 5, 0.01, 4, 1, True, p=3.0, seed=18, nforce=2)], "f64")
    assert ei.value.status == swr.KFP_ENOTSUP
