"""Host-side logic that needs no GPU: the autotuner's cache, the experiment tables,
the problem flags, the model-problem inputs and the benchmark's profile lookup."""
import hashlib
import json
import types

import numpy as np
import pytest

import bench
import oracle
from paper_1306_4596_gb300 import autotune, experiments, inputs, swr


class _FakeBatch:
    def __init__(self, probs):
        self.probs = probs
        self.configured = []

    def configure(self, bps, order, shape=1):
        self.configured.append((bps, order, shape))


def test_autotune_signature_ignores_problem_order_but_not_precision():
    probs = inputs.batch_instances(4)
    a = autotune.signature(probs, "f64")
    assert a == autotune.signature(list(reversed(probs)), "f64")
    assert a != autotune.signature(probs, "f32")
    assert a != autotune.signature(probs[:3], "f64")


def test_autotune_applies_a_cached_choice_without_timing(tmp_path, monkeypatch):
    monkeypatch.setenv("KFP_SWR_CACHE", str(tmp_path))
    probs = inputs.batch_instances(3)
    key = autotune.signature(probs, "f64")
    entry = {"blocks_per_sm": 1, "unit_order": 0, "tile_shape": 2, "ms": 1.5, "candidates": []}
    (tmp_path / "autotune.json").write_text(json.dumps({key: entry}))
    fake = _FakeBatch(probs)
    res = autotune.tune(fake, "f64")
    assert res["cached"] and fake.configured == [(1, 0, 2)]


def test_autotune_candidates_cover_every_tile_shape():
    assert len(autotune.CANDIDATES) >= 8 and len(set(autotune.CANDIDATES)) == len(autotune.CANDIDATES)
    assert {c[2] for c in autotune.CANDIDATES} == set(range(swr.TILE_SHAPES))


def test_table1_formatting():
    rows = [
        {"method": "CSWR", "overlap": 3, "j": 0, "iters": 106, "converged": True},
        {"method": "CSWR", "overlap": 3, "j": 1, "iters": 150, "converged": False},
        {"method": "CSWR", "overlap": 0, "j": 0, "iters": 1, "converged": False},
        {"method": "OSWR(p)", "overlap": 0, "j": 0, "iters": 11, "converged": True},
    ]
    text = experiments.format_table1(rows)
    lines = text.splitlines()
    assert lines[0] == "| decomposition | method | j=0 | j=1 |"
    assert "| overlap 3 cells | CSWR | 106 | >150 |" in lines
    assert "| no overlap | CSWR | - |  |" in lines
    assert "| no overlap | OSWR(p) | 11 |  |" in lines


def test_problem_flags():
    p = inputs.small_robin()
    assert swr.problem_flags(p) == 0
    assert swr.problem_flags(p.replace(gauss_seidel=True)) == swr.KFP_FLAG_GAUSS_SEIDEL
    both = p.replace(neumann_v=True, periodic_x=True, scheme=1)
    assert swr.problem_flags(both) == (swr.KFP_FLAG_NEUMANN_V | swr.KFP_FLAG_PERIODIC_X | swr.KFP_FLAG_SPLIT_SCHEME)


@pytest.mark.parametrize("j", [0, 1])
def test_model_error_equation_setting(j):
    prob = inputs.model_error_equation(j, overlap=3, robin=True, p=4.23, seed=7)
    n = 100 * 2 ** j
    assert (prob.nx, prob.nv, prob.nt) == (n, 2 * n, 2 * n)
    assert prob.dt == prob.hx == pytest.approx(prob.hv)
    assert prob.neumann_v and prob.periodic_x
    assert oracle.validate(prob) == 0  # Courant number exactly 1 at v = +-1 is accepted
    assert np.all(prob.lam0[:, 1] == 0) and np.abs(prob.lam0[:, 0]).max() <= 1
    again = inputs.model_error_equation(j, overlap=3, robin=True, p=4.23, seed=7)
    assert np.array_equal(prob.lam0, again.lam0)
    assert not np.array_equal(prob.lam0, inputs.model_error_equation(j, seed=8).lam0)


def test_profiled_traffic_only_for_the_captured_source(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cuh"
    src.write_bytes(b"// kernel v1\n")
    digest = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    summary = tmp_path / "summary.md"
    summary.write_text(f"source sha256[:16] = {digest}\ntraffic_bytes_per_cell_update stream f64 = 21.5\n"
                       "traffic_bytes_per_cell_update pass f64 = 20.0\n")
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(summary))
    monkeypatch.setattr(bench, "SWEEP_SOURCE", str(src))
    assert bench.profiled_traffic("stream", "f64", 1000) == 21500
    assert bench.profiled_traffic("pass", "f64", 100) == 2000
    assert bench.profiled_traffic("stream", "f32", 1000) is None
    src.write_bytes(b"// kernel v2\n")
    assert bench.profiled_traffic("stream", "f64", 1000) is None


def test_job_rate_and_single_rank_time():
    assert bench.job_rate(2, 1_000, 3, 500.0) == pytest.approx(2 * 1_000 * 3 / 0.5)
    assert bench.max_over_ranks(None, None, 1, 12.5) == 12.5


def test_depth_flag_bits_do_not_overlap_other_flags():
    """KFP_FLAG_DEPTH(n) for n = 1..8 and KFP_FLAG_SHAPE(n) for n = 0..2 sit in bits of
    their own, clear of the single-bit flags."""
    single = (swr.KFP_FLAG_NO_GRAPH | swr.KFP_FLAG_PROFILE | swr.KFP_FLAG_GENERIC | swr.KFP_FLAG_GAUSS_SEIDEL
              | swr.KFP_FLAG_NEUMANN_V | swr.KFP_FLAG_PERIODIC_X | swr.KFP_FLAG_SPLIT_SCHEME
              | swr.KFP_FLAG_PERSISTENT | swr.KFP_FLAG_PER_PASS)
    for n in range(1, swr.MAX_DEPTH + 1):
        d = swr.KFP_FLAG_DEPTH(n)
        assert d & single == 0 and (d >> swr.KFP_FLAG_DEPTH_SHIFT) == n
        for m in range(swr.TILE_SHAPES):
            assert d & swr.KFP_FLAG_SHAPE(m) == 0 and swr.KFP_FLAG_SHAPE(m) & single == 0


def test_committed_mixed_workload_record_is_readable_and_consistent():
    """The bench repeats the committed --mixed-workload record: it parses, both arms
    reached the tolerance, and the speed-up is the ratio of the two times."""
    d = bench.committed_mixed_workload()
    assert d is not None and d["tol"] == 1e-8
    assert d["f64"]["reached"] and d["mixed"]["reached"]
    assert d["f64"]["e_mis"] < d["tol"] and d["mixed"]["e_mis"] < d["tol"]
    assert d["speedup_mixed_vs_f64"] == pytest.approx(d["f64"]["seconds"] / d["mixed"]["seconds"])
    assert "profiles/mixed_precision_workload.md" in d["source"]
