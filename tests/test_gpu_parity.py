"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: FP64 -- max-norm error <= 1e-12 relative to the oracle's max-norm for
the solution, interface data and overlap values; the per-iteration norms e_mis and
e_chg are differences of nearly equal numbers, so they are compared in absolute
terms against 1e-12 times the scale of the values they are taken from.  FP32 --
relative L2 error <= 1e-5 (the FP32 path rounds every step to 24 bits).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1306_4596_gb300 import inputs

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_TOL = 1e-5


def _swr():
    from paper_1306_4596_gb300 import swr
    return swr


def rel_max(a, b):
    scale = max(np.abs(b).max(), 1e-300) if b.size else 1.0
    return np.abs(a - b).max() / scale if a.size else 0.0


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0) if a.size else 0.0


def run_gpu(prob, iters, precision="f64", **kw):
    swr = _swr()
    with swr.SWR(prob, precision, **kw) as s:
        s.sweep(iters)
        out = {"u_T": s.solution(), "lam": s.traces(), "bands": s.bands(), "hist": s.error()[3],
               "stats": s.stats()}
    return out


def run_oracle(prob, iters):
    lam = np.zeros(oracle.trace_shape(prob)) if prob.lam0 is None else prob.lam0.copy()
    if prob.periodic_x:  # node nx repeats node 0, also in the initial interface data
        lam[..., prob.nx] = lam[..., 0]
    hist = []
    bands = None
    u_T = None
    for _ in range(iters):
        new, bands, u_T = oracle.swr_iteration(prob, lam)
        hist.append(oracle.interface_norms(prob, bands, new, lam))
        lam = new
    return {"u_T": u_T, "lam": lam, "bands": bands, "hist": np.array(hist).reshape(iters, 3)}


def check_f64(gpu, ref, prob):
    assert rel_max(gpu["u_T"], ref["u_T"]) <= F64_TOL, rel_max(gpu["u_T"], ref["u_T"])
    if prob.nstrips > 1:
        assert rel_max(gpu["lam"], ref["lam"]) <= F64_TOL, rel_max(gpu["lam"], ref["lam"])
        assert rel_max(gpu["bands"], ref["bands"]) <= F64_TOL, rel_max(gpu["bands"], ref["bands"])
        uscale = max(np.abs(ref["bands"]).max(), 1e-300)
        lscale = max(np.abs(ref["lam"]).max(), np.abs(prob.lam0).max() if prob.lam0 is not None else 0, 1e-300)
        dh = np.abs(gpu["hist"] - ref["hist"])
        assert dh[:, 0].max() <= F64_TOL * uscale, (dh[:, 0], uscale)
        assert dh[:, 1].max() <= F64_TOL * lscale, (dh[:, 1], lscale)
        nband = ref["bands"][:, 0].size
        jtol = F64_TOL * uscale * math.sqrt(prob.dt * prob.hx * nband) * 4
        assert np.abs(np.sqrt(gpu["hist"][:, 2]) - np.sqrt(ref["hist"][:, 2])).max() <= jtol


def check_f32(gpu, ref, prob):
    assert rel_l2(gpu["u_T"], ref["u_T"]) <= F32_TOL, rel_l2(gpu["u_T"], ref["u_T"])
    if prob.nstrips > 1:
        assert rel_l2(gpu["lam"], ref["lam"]) <= F32_TOL, rel_l2(gpu["lam"], ref["lam"])
        assert rel_l2(gpu["bands"], ref["bands"]) <= F32_TOL, rel_l2(gpu["bands"], ref["bands"])


RD = inputs.random_data
SMALL_CASES = [
    # (label, problem factory, iterations).  One forcing term (time-dependent or
    # constant) and no forcing run the TMA-fed sweep; two terms run the plain one.
    ("small_dirichlet", inputs.small_dirichlet, 6),
    ("small_robin", inputs.small_robin, 6),
    ("dirichlet_S3_ov2", lambda: RD(37, 24, 7, 0.01, 3, 2, False, seed=1, nforce=1), 3),
    ("robin_S4_ov0_pq", lambda: RD(61, 32, 5, 0.01, 4, 0, True, p=3.0, q=1.5, seed=2, nforce=1), 3),
    ("robin_S2_ov3_one_warp", lambda: RD(29, 16, 4, 0.02, 2, 3, True, p=2.0, seed=3, nforce=1), 3),
    ("robin_ragged_31_cols", lambda: RD(30, 16, 4, 0.02, 2, 1, True, p=2.0, seed=4, nforce=1), 3),
    ("two_columns", lambda: RD(1, 8, 3, 0.2, 2, 1, False, seed=5, nforce=1), 3),
    ("max_overlap", lambda: RD(95, 60, 6, 0.005, 5, 11, True, p=5.0, seed=6, nforce=1), 3),
    ("robin_max_overlap_odd", lambda: RD(64, 30, 5, 0.005, 3, 9, True, p=5.0, q=2.0, seed=7, nforce=1), 3),
    ("single_step", lambda: RD(40, 16, 1, 0.01, 2, 2, True, seed=8, nforce=1), 2),
    ("dirichlet_no_overlap", lambda: RD(33, 16, 4, 0.01, 2, 0, False, seed=9, nforce=1), 3),
    ("single_strip", lambda: RD(70, 32, 5, 0.01, 1, 0, False, seed=10, nforce=1), 1),
    ("no_forcing", lambda: RD(150, 40, 7, 0.005, 4, 2, True, p=3.0, seed=16, nforce=0), 3),
    ("constant_forcing", lambda: RD(200, 64, 9, 0.004, 4, 0, True, p=3.0, seed=17, nforce=1,
                                    constant_in_time=True), 3),
    ("two_forcing_terms", lambda: RD(61, 32, 5, 0.01, 4, 1, True, p=3.0, seed=18, nforce=2), 3),
    ("long_strips_many_chunks", lambda: RD(250, 400, 6, 2e-4, 2, 3, True, p=6.0, seed=19, nforce=1,
                                           v_range=(-2.0, 2.0)), 2),
    # zero boundary data and long strips: interior chunks take the branch-free path
    ("fast_dirichlet_ov3", lambda: RD(90, 256, 6, 0.002, 2, 3, False, seed=20, nforce=1, boundary_data=False), 3),
    ("fast_robin_pq_time_forcing", lambda: RD(77, 192, 5, 0.002, 3, 0, True, p=4.0, q=2.0, seed=21, nforce=1,
                                              boundary_data=False), 3),
    ("fast_no_forcing_ov5", lambda: RD(64, 128, 5, 0.003, 2, 5, True, p=3.0, seed=22, nforce=0,
                                       boundary_data=False), 3),
    ("fast_const_forcing_S3", lambda: RD(120, 300, 4, 0.002, 3, 4, True, p=5.0, seed=23, nforce=1,
                                         constant_in_time=True, boundary_data=False), 3),
    # strips whose row count is a multiple of 16 (the last chunk is full and holds an end
    # row) and strips of exactly one chunk (both end rows in it)
    ("fast_full_last_chunk_robin", lambda: RD(90, 250, 6, 0.002, 2, 3, True, p=4.0, seed=24, nforce=1,
                                              boundary_data=False), 3),
    ("fast_full_last_chunk_dirichlet", lambda: RD(90, 250, 6, 0.002, 2, 3, False, seed=25, nforce=1,
                                                  boundary_data=False), 3),
    ("fast_one_chunk_strips_robin", lambda: RD(70, 60, 5, 0.004, 4, 0, True, p=3.0, q=2.0, seed=26, nforce=1,
                                               boundary_data=False), 3),
    ("fast_one_chunk_strips_dirichlet", lambda: RD(70, 60, 5, 0.004, 4, 0, False, seed=27, nforce=0,
                                                   boundary_data=False), 3),
    ("bumps_8_strips", lambda: inputs.gaussian_bumps(300, 512, 40, 8e-4, 8, p=4.0, seed=11), 2),
    ("bumps_dirichlet_ov4", lambda: inputs.gaussian_bumps(130, 256, 30, 1.5e-3, 4, seed=12, overlap=4,
                                                          robin=False), 2),
]


@pytest.mark.parametrize("label,factory,iters", SMALL_CASES, ids=[c[0] for c in SMALL_CASES])
def test_f64_matches_oracle(label, factory, iters):
    prob = factory()
    ref = run_oracle(prob, iters) if prob.nstrips > 1 else {"u_T": oracle.monolithic(prob)}
    gpu = run_gpu(prob, iters)
    check_f64(gpu, ref, prob)


@pytest.mark.parametrize("label,factory,iters", SMALL_CASES, ids=[c[0] for c in SMALL_CASES])
def test_f32_matches_oracle(label, factory, iters):
    prob = factory()
    ref = run_oracle(prob, iters) if prob.nstrips > 1 else {"u_T": oracle.monolithic(prob)}
    gpu = run_gpu(prob, iters, "f32")
    check_f32(gpu, ref, prob)


@pytest.mark.parametrize("label,factory,iters", SMALL_CASES[:6] + SMALL_CASES[12:14],
                         ids=[c[0] for c in SMALL_CASES[:6] + SMALL_CASES[12:14]])
def test_f64_plain_kernel_matches_oracle(label, factory, iters):
    """The plain (non-TMA) sweep kernel on the cases the TMA-fed one normally takes."""
    prob = factory()
    ref = run_oracle(prob, iters) if prob.nstrips > 1 else {"u_T": oracle.monolithic(prob)}
    check_f64(run_gpu(prob, iters, generic=True), ref, prob)


def test_f64_without_graph_is_bitwise_identical():
    prob = inputs.random_data(61, 32, 5, 0.01, 4, 2, True, p=3.0, seed=13)
    a = run_gpu(prob, 3)
    b = run_gpu(prob, 3, graph=False)
    for key in ("u_T", "lam", "bands", "hist"):
        assert np.array_equal(a[key], b[key]), key


def test_converged_gpu_equals_single_domain():
    """Pin 3 on the GPU path: the converged iterate equals the single-domain solve."""
    prob = inputs.manufactured(64, 64, 20, 0.1, nstrips=2, overlap=0, robin=True, p=8.0)
    mono = oracle.monolithic(prob)
    swr = _swr()
    with swr.SWR(prob) as s:
        n = s.sweep(300, 1e-14, 0)
        u = s.solution()
    assert n < 300
    assert np.abs(u - mono).max() <= 1e-11


def test_full_grid_of_the_at_scale_workload():
    """The 2048 x 4096, 8-strip grid in the benchmark's launch configuration, on a
    short window the oracle finishes in seconds (nt = 8)."""
    prob = inputs.at_scale().replace(nt=8)
    prob.f_time = prob.f_time[:, :9].copy()
    ref = run_oracle(prob, 2)
    check_f64(run_gpu(prob, 2), ref, prob)
    check_f32(run_gpu(prob, 2, "f32"), ref, prob)


def test_at_scale_properties():
    """Full benchmark workload (2 iterations): deterministic, non-negative (maximum
    principle with non-negative data), and resumable bit for bit from the exported
    interface data."""
    swr = _swr()
    prob = inputs.at_scale()
    with swr.SWR(prob) as s:
        s.sweep(1)
        lam1 = s.traces()
        s.sweep(1)
        u_a = s.solution()
        hist_a = s.error()[3]
    assert np.isfinite(u_a).all() and u_a.min() >= -1e-14
    assert hist_a[1, 0] < hist_a[0, 0]
    p2 = inputs.at_scale()
    p2.lam0 = lam1
    with swr.SWR(p2) as s:
        s.sweep(1)
        u_b = s.solution()
        hist_b = s.error()[3]
    assert np.array_equal(u_a, u_b)
    assert np.array_equal(hist_a[1], hist_b[0])


def test_resume_from_set_traces():
    swr = _swr()
    prob = inputs.random_data(45, 24, 6, 0.01, 3, 1, True, p=2.0, seed=14)
    with swr.SWR(prob) as s:
        s.sweep(4)
        ref = s.traces()
        hist = s.error()[3]
    with swr.SWR(prob) as s:
        s.sweep(2)
        ck = s.traces()
    with swr.SWR(prob) as s:
        s.set_traces(ck)
        s.sweep(2)
        assert np.array_equal(s.traces(), ref)
        assert np.array_equal(s.error()[3], hist[2:])


@pytest.mark.parametrize("factory", [inputs.small_dirichlet, inputs.small_robin], ids=["dirichlet", "robin"])
def test_tolerance_stops_and_reports(factory):
    """The small workload iterated until the interface change is below 1e-10 (or 50
    iterations): the same count as the oracle, and the final iterate matches it."""
    swr = _swr()
    prob = factory()
    ref = oracle.swr_solve(prob, 50, 1e-10, 0)
    with swr.SWR(prob) as s:
        n = s.sweep(50, 1e-10, 0)
        assert n == ref["iters"]  # 29 (Dirichlet, overlap 4); the 50-iteration cap (Robin p = 2)
        u = s.solution()
        assert np.abs(u - ref["u_T"]).max() <= 1e-12 * np.abs(ref["u_T"]).max()
        with pytest.raises(swr.KfpError) as ei:
            swr.kfp_swr_sweep(s.h, 2, 1e-30, 1)
        assert ei.value.status == swr.KFP_ENOTCONV


def test_nan_input_is_reported():
    swr = _swr()
    prob = inputs.small_robin()
    prob.u0 = prob.u0.copy()
    prob.u0[10, 10] = np.nan
    with swr.SWR(prob) as s:
        with pytest.raises(swr.KfpError) as ei:
            swr.kfp_swr_sweep(s.h, 2, 1e-8, 1)
        assert ei.value.status == swr.KFP_ENUMERIC


def test_host_inputs_match_device_inputs():
    prob = inputs.random_data(50, 24, 5, 0.01, 3, 2, True, p=2.0, seed=15)
    a = run_gpu(prob, 2, inputs_on="host")
    b = run_gpu(prob, 2, inputs_on="device")
    for key in ("u_T", "lam", "bands", "hist"):
        assert np.array_equal(a[key], b[key]), key


GS_CASES = [
    ("small_dirichlet", inputs.small_dirichlet, 4),
    ("small_robin", inputs.small_robin, 4),
    ("robin_4_strips_ov2_fast", lambda: RD(90, 256, 6, 0.002, 4, 2, True, p=5.0, seed=50, nforce=1,
                                           boundary_data=False), 3),
    ("dirichlet_3_strips_bc_data", lambda: RD(37, 24, 7, 0.01, 3, 2, False, seed=51, nforce=1), 3),
    ("robin_two_terms_plain_kernel", lambda: RD(61, 32, 5, 0.01, 4, 0, True, p=3.0, q=1.5, seed=52, nforce=2), 3),
]


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("label,factory,iters", GS_CASES, ids=[c[0] for c in GS_CASES])
def test_gauss_seidel_order_matches_oracle(label, factory, iters, precision):
    prob = factory().replace(gauss_seidel=True)
    ref = run_oracle(prob, iters)
    gpu = run_gpu(prob, iters, precision)
    (check_f64 if precision == "f64" else check_f32)(gpu, ref, prob)


# Model-problem boundary conditions (Section 6.1): zero flux in v and/or periodic x.
# Column counts put node nx on the first, a middle and the last output lane of a warp
# (nx = 30, 89, 29 / 119) and at the smallest periodic grid (nx = 2).
VARIANT_CASES = [
    ("both_fast_S4_ov0", lambda: RD(119, 256, 6, 0.002, 4, 0, True, p=5.0, seed=60, nforce=1), 3, True, True),
    ("both_fast_S2_ov3_const", lambda: RD(89, 192, 5, 0.002, 2, 3, True, p=4.0, seed=61, nforce=1,
                                          constant_in_time=True), 3, True, True),
    ("both_no_forcing_dirichlet", lambda: RD(30, 128, 5, 0.003, 2, 4, False, seed=62, nforce=0), 3, True, True),
    ("both_two_terms_plain_kernel", lambda: RD(29, 32, 5, 0.01, 4, 0, True, p=3.0, q=1.5, seed=63,
                                               nforce=2), 3, True, True),
    ("both_nx2_single_strip", lambda: RD(2, 16, 4, 0.01, 1, 0, False, seed=64, nforce=1), 1, True, True),
    ("neumann_with_inflow_data", lambda: RD(61, 64, 5, 0.005, 4, 2, True, p=3.0, seed=65, nforce=1), 3,
     True, False),
    ("periodic_with_v_data", lambda: RD(121, 96, 5, 0.004, 3, 1, False, seed=66, nforce=1), 3, False, True),
    ("bumps_both_8_strips", lambda: inputs.gaussian_bumps(300, 512, 40, 8e-4, 8, p=4.0, seed=67), 2, True, True),
]


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("label,factory,iters,neumann,periodic", VARIANT_CASES, ids=[c[0] for c in VARIANT_CASES])
def test_model_problem_boundaries_match_oracle(label, factory, iters, neumann, periodic, precision):
    prob = factory().replace(neumann_v=neumann, periodic_x=periodic)
    ref = run_oracle(prob, iters)
    gpu = run_gpu(prob, iters, precision)
    (check_f64 if precision == "f64" else check_f32)(gpu, ref, prob)
    if periodic:  # node nx repeats node 0 exactly
        assert np.array_equal(gpu["u_T"][:, prob.nx], gpu["u_T"][:, 0])


@pytest.mark.parametrize("label,factory,iters,neumann,periodic", VARIANT_CASES[:3] + VARIANT_CASES[5:7],
                         ids=[c[0] for c in VARIANT_CASES[:3] + VARIANT_CASES[5:7]])
def test_model_problem_boundaries_plain_kernel(label, factory, iters, neumann, periodic):
    prob = factory().replace(neumann_v=neumann, periodic_x=periodic)
    check_f64(run_gpu(prob, iters, "f64", generic=True), run_oracle(prob, iters), prob)


def test_model_problem_gauss_seidel():
    prob = RD(119, 256, 6, 0.002, 4, 0, True, p=5.0, seed=68, nforce=1).replace(
        neumann_v=True, periodic_x=True, gauss_seidel=True)
    check_f64(run_gpu(prob, 3), run_oracle(prob, 3), prob)


def test_model_problem_conserves_mass_on_gpu():
    """Zero flux in v and periodic x: the converged GPU iterate keeps the discrete mass
    of u0 (trapezoid weights in v, the nx unique columns in x) to rounding."""
    prob = inputs.gaussian_bumps(240, 512, 60, 6e-4, 4, p=4.0, seed=69)
    prob = prob.replace(neumann_v=True, periodic_x=True, f_time=np.zeros_like(prob.f_time))
    w = np.full(prob.nv + 1, prob.hv)
    w[0] = w[-1] = 0.5 * prob.hv
    mass = lambda u: float(w @ u[:, : prob.nx].sum(axis=1)) * prob.hx
    swr = _swr()
    with swr.SWR(prob, "f64") as s:
        s.sweep(200, tol=1e-10)
        u_T = s.solution()
    m0 = mass(prob.u0)
    assert abs(mass(u_T) - m0) <= 1e-11 * abs(m0)


# The paper's own scheme (Section 6.2): Lie splitting with P1 elements in v, on the
# model problem (zero flux in v, periodic x).
SPLIT_CASES = [
    ("split_robin_S4_ov0", lambda: RD(61, 64, 5, 0.005, 4, 0, True, p=3.0, q=1.5, seed=70, nforce=1), 3),
    ("split_robin_S2_ov3", lambda: RD(89, 96, 6, 0.004, 2, 3, True, p=4.0, seed=71, nforce=2), 3),
    ("split_dirichlet_S3_ov2", lambda: RD(30, 48, 5, 0.005, 3, 2, False, seed=72, nforce=0), 3),
    ("split_robin_S4_ov1_pq", lambda: RD(119, 128, 4, 0.003, 4, 1, True, p=5.0, q=2.0, seed=73, nforce=1), 3),
    ("split_single_strip", lambda: RD(29, 32, 6, 0.01, 1, 0, False, seed=74, nforce=1), 1),
    ("split_bumps_8_strips", lambda: inputs.gaussian_bumps(300, 512, 40, 8e-4, 8, p=4.0, seed=75), 2),
]


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("label,factory,iters", SPLIT_CASES, ids=[c[0] for c in SPLIT_CASES])
def test_split_scheme_matches_oracle(label, factory, iters, precision):
    prob = factory().replace(neumann_v=True, periodic_x=True, scheme=1)
    ref = run_oracle(prob, iters)
    gpu = run_gpu(prob, iters, precision)
    (check_f64 if precision == "f64" else check_f32)(gpu, ref, prob)
    assert np.array_equal(gpu["u_T"][:, prob.nx], gpu["u_T"][:, 0])


def test_split_scheme_serial_order():
    prob = RD(89, 96, 6, 0.004, 3, 3, True, p=4.0, seed=76, nforce=1).replace(
        neumann_v=True, periodic_x=True, scheme=1, gauss_seidel=True)
    check_f64(run_gpu(prob, 3), run_oracle(prob, 3), prob)


def test_split_scheme_converges_to_single_domain():
    prob = inputs.gaussian_bumps(120, 256, 30, 1.5e-3, 4, p=4.0, seed=77, overlap=2).replace(
        neumann_v=True, periodic_x=True, scheme=1)
    mono = oracle.monolithic(prob)
    swr = _swr()
    with swr.SWR(prob, "f64") as s:
        s.sweep(300, tol=1e-13)
        u = s.solution()
    assert np.abs(u - mono).max() <= 1e-11 * np.abs(mono).max()


@pytest.mark.parametrize("precision", ["f64", "f32", "mixed"])
@pytest.mark.parametrize("overlap", [0, 2])
def test_split_scheme_set_robin_equals_fresh_handle(overlap, precision):
    """New Robin parameters on a live split-scheme handle reach both the elimination
    (its pre-scaled factors) and the back-substitution: the results equal, bit for
    bit, those of a handle created with the new parameters."""
    swr = _swr()
    prob = RD(89, 128, 5, 0.003, 4, overlap, True, p=4.0, seed=78, nforce=1).replace(
        neumann_v=True, periodic_x=True, scheme=1)
    newp, newq = np.array([2.0, 7.0, 3.0]), np.array([5.0, 1.5, 2.5])
    with swr.SWR(prob, precision) as s:
        s.sweep(2)
        s.set_robin(newp, newq)
        s.set_traces(prob.lam0)
        s.sweep(3)
        a = (s.solution(), s.traces())
    fresh = prob.replace()
    fresh.p, fresh.q = newp, newq
    with swr.SWR(fresh, precision) as s:
        s.sweep(3)
        b = (s.solution(), s.traces())
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    if precision == "f64":
        ref = run_oracle(fresh, 3)
        assert rel_max(a[0], ref["u_T"]) <= F64_TOL and rel_max(a[1], ref["lam"]) <= F64_TOL


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("label,factory,iters", [SPLIT_CASES[0], SPLIT_CASES[3], SPLIT_CASES[5]],
                         ids=[SPLIT_CASES[0][0], SPLIT_CASES[3][0], SPLIT_CASES[5][0]])
def test_split_scheme_tile_shapes_are_bitwise_identical(label, factory, iters, precision):
    """The TMA-fed split-scheme pass gives the same bits in every tile shape (16- or
    8-row ring stages; its branch-free and row-by-row paths do the same arithmetic)."""
    prob = factory().replace(neumann_v=True, periodic_x=True, scheme=1)
    ref = run_gpu(prob, iters, precision, tile_shape=0)
    for shape in (1, 2):
        out = run_gpu(prob, iters, precision, tile_shape=shape)
        for key in ("u_T", "lam", "bands", "hist"):
            assert np.array_equal(out[key], ref[key]), (shape, key)


@pytest.mark.parametrize("label,factory,iters", [SPLIT_CASES[0], SPLIT_CASES[2], SPLIT_CASES[5]],
                         ids=[SPLIT_CASES[0][0], SPLIT_CASES[2][0], SPLIT_CASES[5][0]])
def test_split_scheme_plain_kernel_matches_oracle(label, factory, iters):
    """The plain-load split-scheme pass (taken for two or more forcing terms and with
    KFP_FLAG_GENERIC) on cases the TMA-fed one normally runs."""
    prob = factory().replace(neumann_v=True, periodic_x=True, scheme=1)
    check_f64(run_gpu(prob, iters, "f64", generic=True), run_oracle(prob, iters), prob)
