"""The C-ABI library builds, loads and exports every entry point declared in
include/*.h; host-side validation answers without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1306_4596_gb300 import build, inputs, swr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(inc, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(kfp_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("kfp_swr_create", "kfp_swr_sweep", "kfp_swr_traces", "kfp_swr_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.build())
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(swr.EXPORTED) <= declared_functions()


def _desc(prob, **kw):
    d = swr.kfp_swr_desc(prob.x0, prob.x1, prob.v0, prob.v1, prob.dt, prob.nx, prob.nv, prob.nt,
                         prob.nstrips, prob.overlap, int(prob.robin), None, None, 0, 0)
    for k, v in kw.items():
        setattr(d, k, v)
    return d


def _create_status(desc, prob):
    lib = swr.load()
    u0 = np.ascontiguousarray(prob.u0)
    pb = swr.kfp_swr_problem(0, u0.ctypes.data, 0, None, None, None, None, None)
    out = ctypes.c_void_p(123)
    st = lib.kfp_swr_create(ctypes.byref(desc), ctypes.byref(pb), None, ctypes.byref(out))
    return st, out.value, lib.kfp_swr_create_error().decode()


def test_validation_without_gpu():
    prob = inputs.small_dirichlet()
    st, h, msg = _create_status(_desc(prob, dt=0.05), prob)
    assert st == swr.KFP_ECFL and h is None and "CFL" in msg
    st, h, msg = _create_status(_desc(prob, nstrips=3), prob)
    assert st == swr.KFP_EINVAL and h is None and "divide" in msg
    st, h, msg = _create_status(_desc(prob, overlap_cells=32), prob)
    assert st == swr.KFP_EINVAL and "overlap" in msg
    st, h, msg = _create_status(_desc(prob, tc=swr.KFP_ROBIN), prob)  # Robin without p
    assert st == swr.KFP_EINVAL and "p" in msg
    p = np.array([-1.0])
    st, h, msg = _create_status(_desc(prob, tc=swr.KFP_ROBIN, p=p.ctypes.data), prob)
    assert st == swr.KFP_EINVAL and "> 0" in msg
    st, h, msg = _create_status(_desc(prob, nx=0), prob)
    assert st == swr.KFP_EINVAL
    # the split scheme of Section 6.2 is built for the model problem only
    st, h, msg = _create_status(_desc(prob, flags=swr.KFP_FLAG_SPLIT_SCHEME), prob)
    assert st == swr.KFP_EINVAL and h is None and "split" in msg
    st, h, msg = _create_status(_desc(prob, flags=swr.KFP_FLAG_SPLIT_SCHEME | swr.KFP_FLAG_NEUMANN_V), prob)
    assert st == swr.KFP_EINVAL and "split" in msg
    tiny = inputs.random_data(1, 8, 2, 0.1, 2, 1, False, seed=0)
    st, h, msg = _create_status(_desc(tiny, flags=swr.KFP_FLAG_PERIODIC_X), tiny)
    assert st == swr.KFP_EINVAL and "periodic" in msg


def test_null_arguments_are_rejected():
    lib = swr.load()
    assert lib.kfp_swr_create(None, None, None, None) == swr.KFP_EINVAL
    assert lib.kfp_swr_sweep(None, 1, 0.0, 0, None) == swr.KFP_EINVAL
    assert lib.kfp_swr_traces(None, 0, 0, None, 0) == swr.KFP_EINVAL
    assert lib.kfp_swr_error(None, None, None, None, None, 0) == swr.KFP_EINVAL
    assert lib.kfp_swr_pipeline_stats(None, None, None, None, None, None) == swr.KFP_EINVAL
    assert lib.kfp_swr_stats(None, None, None, None, None, None, None) == swr.KFP_EINVAL
    lib.kfp_swr_destroy(None)
    assert lib.kfp_swr_last_error(None) == b""


def test_cell_update_count():
    assert swr.cell_updates_per_iteration(inputs.small_dirichlet()) == 65 * (35 + 35) * 20
    assert swr.cell_updates_per_iteration(inputs.small_robin()) == 65 * (33 + 33) * 20
    big = inputs.Problem(0, 1, -4, 4, 1e-4, 2048, 4096, 2000, 8, 0, True, np.full(7, 4.0), np.full(7, 4.0),
                         np.zeros((1, 1)), np.zeros((1, 1)), np.zeros((1, 1, 1)))
    assert swr.cell_updates_per_iteration(big) == 2049 * (8 * 513) * 2000
