"""Pipelined iterates (several consecutive SWR iterates swept in one streamed launch,
as a wavefront over iterate and time step) against one iterate at a time.

Iterate d of a group solves time step k once iterate d-1 has recorded the interface
data at t^k and t^(k+1); every iterate runs the arithmetic of a lone iteration in the
same order, so the results, the error history and the iteration count at a tolerance
must agree bit for bit with the single-iterate form, whose parity with the oracle is
checked in tests/test_gpu_parity.py (which also runs the pipelined form on the full
at-scale grid, chosen there by default).
"""
import numpy as np
import pytest

import oracle
from paper_1306_4596_gb300 import inputs

pytestmark = pytest.mark.gpu

RD = inputs.random_data


def _run(prob, iters, precision="f64", tol=0.0, tol_kind=0, cont=0, **kw):
    from paper_1306_4596_gb300 import swr
    with swr.SWR(prob, precision, **kw) as s:
        n = s.sweep(iters, tol, tol_kind)
        if cont:
            s.sweep(cont)
        return {"n": n, "u_T": s.solution(), "lam": s.traces(), "bands": s.bands(), "hist": s.error()[3],
                "pipe": s.pipeline_stats(), "cnt": s.counters()}


def _same(a, b):
    for key in ("u_T", "lam", "bands", "hist"):
        assert np.array_equal(a[key], b[key]), key


CASES = [
    ("small_robin", inputs.small_robin, 5),
    ("small_dirichlet", inputs.small_dirichlet, 5),
    ("three_passes", lambda: RD(61, 32, 3, 0.01, 4, 0, True, p=3.0, q=1.5, seed=81, nforce=1), 5),
    ("robin_time_forcing", lambda: RD(77, 192, 7, 0.002, 3, 0, True, p=4.0, q=2.0, seed=82, nforce=1,
                                      boundary_data=False), 5),
    ("const_forcing_ov4", lambda: RD(250, 300, 6, 0.002, 3, 4, True, p=5.0, seed=83, nforce=1,
                                     constant_in_time=True, boundary_data=False), 5),
    ("no_forcing_dirichlet", lambda: RD(150, 128, 5, 0.003, 2, 4, False, seed=84, nforce=0), 5),
    ("bumps_8_strips", lambda: inputs.gaussian_bumps(300, 512, 40, 8e-4, 8, p=4.0, seed=85), 5),
]


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("label,factory,iters", CASES, ids=[c[0] for c in CASES])
def test_depths_equal_single_iterates(label, factory, iters, precision):
    """Groups of 2, 3, 4 and 8 (with partial groups: 5 iterations) give the bits of one
    iterate at a time."""
    prob = factory()
    ref = _run(prob, iters, precision, depth=1)
    assert ref["pipe"]["depth"] == 1
    for D in (2, 3, 4, 8):
        got = _run(prob, iters, precision, depth=D)
        _same(ref, got)
        eff = min(D, prob.nt - 1) if prob.nt >= 3 else 1
        assert got["pipe"]["depth"] == eff
        if eff > 1:
            groups = iters // eff + (1 if iters % eff >= 2 else 0)
            assert got["pipe"]["stream_launches"] == groups


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("shape", [0, 2])
def test_depth_with_other_tile_shapes(shape, precision):
    prob = CASES[6][1]()
    ref = _run(prob, 4, precision, depth=1)
    _same(ref, _run(prob, 4, precision, depth=4, tile_shape=shape))


@pytest.mark.parametrize("tol_kind", [0, 1])
def test_tolerance_stop_inside_a_group(tol_kind):
    """A tolerance met by the second iterate of a group of four: the same count and
    state as one iterate at a time, and the sweep continues from that iterate."""
    prob = RD(90, 256, 12, 0.002, 4, 2, True, p=5.0, seed=88, nforce=1, boundary_data=False)
    full = _run(prob, 12, depth=1)
    col = 1 if tol_kind == 0 else 0
    v = full["hist"][:, col]
    assert v[5] < v[:5].min(), v
    tol = 0.5 * (v[5] + v[:5].min())  # first met by iteration 6 = second iterate of the second group
    a = _run(prob, 40, tol=tol, tol_kind=tol_kind, cont=3, depth=1)
    b = _run(prob, 40, tol=tol, tol_kind=tol_kind, cont=3, depth=4)
    assert a["n"] == b["n"] == 6
    _same(a, b)


def test_mixed_precision_correction_solver_pipelined():
    """The FP32 correction solver of the mixed-precision form in groups of four: the
    same correction iterates, stopping decisions and results as one at a time."""
    prob = inputs.gaussian_bumps(128, 256, 60, 1.6e-3, 8, p=4.0, seed=89)
    from paper_1306_4596_gb300 import swr
    out = []
    for D in (1, 4):
        with swr.SWR(prob, "mixed", depth=D) as s:
            n = s.sweep(8, 1e-10, 1)
            out.append({"n": n, "u_T": s.solution(), "lam": s.traces(), "bands": s.bands(),
                        "hist": s.error()[3], "cnt": s.counters()})
    _same(out[0], out[1])
    assert out[0]["n"] == out[1]["n"]
    assert out[0]["cnt"]["fp32_iterations"] == out[1]["cnt"]["fp32_iterations"]
    assert out[0]["hist"][-1, 0] < 1e-10


def test_pipelined_matches_oracle_three_iterations():
    """The pipelined form against the oracle directly (groups of 3 on 8 strips)."""
    prob = inputs.gaussian_bumps(200, 400, 12, 1e-3, 8, p=4.0, seed=90)
    got = _run(prob, 3, depth=3)
    assert got["pipe"]["depth"] == 3 and got["pipe"]["stream_launches"] == 1
    lam = prob.lam0
    for _ in range(3):
        lam, bands, u_T = oracle.swr_iteration(prob, lam)
    assert np.abs(got["u_T"] - u_T).max() <= 1e-12 * np.abs(u_T).max()
    assert np.abs(got["lam"] - lam).max() <= 1e-12 * np.abs(lam).max()


def test_default_depth_fills_the_device_on_the_at_scale_grid():
    """On the 2048 x 4096, 8-strip grid (144 units per pass) the library chooses to
    pipeline iterates by default; the explicit launch forms do not."""
    from paper_1306_4596_gb300 import swr
    prob = inputs.at_scale().replace(nt=8)
    prob.f_time = prob.f_time[:, :9].copy()
    with swr.SWR(prob) as s:
        assert s.pipeline_stats()["depth"] >= 2
    with swr.SWR(prob, persistent=False) as s:
        assert s.pipeline_stats()["depth"] == 1
    with swr.SWR(prob, persistent=True) as s:
        assert s.pipeline_stats()["depth"] == 1


# The paper's model problem (zero flux in v, periodic x; Section 6.1), with this
# library's scheme and with the split P1 scheme of Section 6.2: the periodic column
# wrap runs between passes, so groups run one launch per slot (grid.z = iterate).
MODEL_CASES = [
    ("model_robin_S4", lambda: RD(119, 256, 6, 0.002, 4, 0, True, p=5.0, seed=60, nforce=1), 0),
    ("model_dirichlet_ov4", lambda: RD(30, 128, 5, 0.003, 2, 4, False, seed=62, nforce=0), 0),
    ("model_bumps_8_strips", lambda: inputs.gaussian_bumps(300, 512, 40, 8e-4, 8, p=4.0, seed=67), 0),
    ("split_robin_S4_pq", lambda: RD(61, 64, 5, 0.005, 4, 0, True, p=3.0, q=1.5, seed=70, nforce=1), 1),
    ("split_robin_S4_ov1", lambda: RD(119, 128, 4, 0.003, 4, 1, True, p=5.0, q=2.0, seed=73, nforce=1), 1),
    ("split_bumps_8_strips", lambda: inputs.gaussian_bumps(300, 512, 40, 8e-4, 8, p=4.0, seed=75), 1),
]


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("label,factory,scheme", MODEL_CASES, ids=[c[0] for c in MODEL_CASES])
def test_slot_launched_groups_equal_single_iterates(label, factory, scheme, precision):
    prob = factory().replace(neumann_v=True, periodic_x=True, scheme=scheme)
    ref = _run(prob, 5, precision, depth=1)
    for D in (2, 3, 4):
        got = _run(prob, 5, precision, depth=D)
        _same(ref, got)
        assert got["pipe"]["depth"] == min(D, prob.nt - 1)
        assert got["pipe"]["stream_launches"] == 0  # one launch per slot, no streamed launch
    assert np.array_equal(ref["u_T"][:, prob.nx], ref["u_T"][:, 0])


@pytest.mark.parametrize("scheme", [0, 1])
def test_slot_launched_groups_stop_inside_a_group(scheme):
    prob = RD(90, 256, 12, 0.002, 4, 2, True, p=5.0, seed=88, nforce=1, boundary_data=False).replace(
        neumann_v=True, periodic_x=True, scheme=scheme)
    v = _run(prob, 12, depth=1)["hist"][:, 1]
    assert v[5] < v[:5].min(), v
    tol = 0.5 * (v[5] + v[:5].min())
    a = _run(prob, 40, tol=tol, cont=3, depth=1)
    b = _run(prob, 40, tol=tol, cont=3, depth=4)
    assert a["n"] == b["n"] == 6
    _same(a, b)


@pytest.mark.parametrize("scheme", [0, 1])
def test_mixed_precision_model_problem_pipelined(scheme):
    """The FP32 correction solver on the model problem, in slot-launched groups."""
    prob = inputs.gaussian_bumps(128, 256, 60, 1.6e-3, 8, p=4.0, seed=91).replace(
        neumann_v=True, periodic_x=True, scheme=scheme)
    from paper_1306_4596_gb300 import swr
    out = []
    for D in (1, 4):
        with swr.SWR(prob, "mixed", depth=D) as s:
            n = s.sweep(8, 1e-10, 1)
            out.append({"n": n, "u_T": s.solution(), "lam": s.traces(), "bands": s.bands(),
                        "hist": s.error()[3], "cnt": s.counters()})
    _same(out[0], out[1])
    assert out[0]["cnt"]["fp32_iterations"] == out[1]["cnt"]["fp32_iterations"]
