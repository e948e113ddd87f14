"""Plain FP64 CPU oracle for Schwarz waveform relaxation on the Kolmogorov equation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product package (``paper_1306_4596_gb300``) never imports it and shares no code
with it; the two meet only through the seeded inputs of
``paper_1306_4596_gb300.inputs``.

The arithmetic lives in ``kfp_oracle.c`` (plain C, FP64, single thread, plain
Thomas per column and step).  This module compiles it with gcc on first use and
binds it with ctypes.  Every function cites the paper passage it follows in the
C source; the Python side only marshals numpy arrays.

Parity status: every function is pinned by the CPU tests in
``tests/test_oracle_pins.py`` (closed-form Kolmogorov Gaussian, manufactured
solutions, exact discrete eigen-solution, dense space-time brute force, the
monolithic fixed point and the contraction invariants of Sections 4 and 5).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kfp_oracle.c")
_HDR = os.path.join(_HERE, "kfp_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libkfp_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class _Desc(ctypes.Structure):
    _fields_ = [
        ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("v0", ctypes.c_double), ("v1", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("nx", ctypes.c_int), ("nv", ctypes.c_int), ("nt", ctypes.c_int),
        ("nstrips", ctypes.c_int), ("overlap", ctypes.c_int), ("robin", ctypes.c_int),
        ("p", _dp), ("q", _dp), ("gauss_seidel", ctypes.c_int), ("neumann_v", ctypes.c_int),
        ("periodic_x", ctypes.c_int), ("scheme", ctypes.c_int),
    ]


class _Problem(ctypes.Structure):
    _fields_ = [
        ("u0", _dp), ("nforce", ctypes.c_int), ("f_time", _dp), ("f_space", _dp),
        ("bc_xin", _dp), ("bc_v", _dp),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, so that x86 and Arm round alike)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.kfo_validate.argtypes = [ctypes.POINTER(_Desc)]
            lib.kfo_strip_layout.argtypes = [ctypes.POINTER(_Desc), _ip, _ip]
            lib.kfo_swr_iteration.argtypes = [ctypes.POINTER(_Desc), ctypes.POINTER(_Problem),
                                              _dp, _dp, _dp, _dp]
            lib.kfo_interface_norms.argtypes = [ctypes.POINTER(_Desc), _dp, _dp, _dp, _dp, _dp, _dp]
            lib.kfo_swr_solve.argtypes = [ctypes.POINTER(_Desc), ctypes.POINTER(_Problem), _dp,
                                          ctypes.c_int, ctypes.c_double, ctypes.c_int, _ip, _dp, _dp]
            lib.kfo_monolithic.argtypes = [ctypes.POINTER(_Desc), ctypes.POINTER(_Problem), _dp, _dp]
            lib.kfo_thomas.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
            lib.kfo_swr_adjoint.argtypes = [ctypes.POINTER(_Desc), ctypes.POINTER(_Problem), _dp, ctypes.c_int,
                                            _dp, _dp, _dp]
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


class _Marshalled:
    """Keeps the numpy buffers alive while the C structs point at them."""

    def __init__(self, prob, nstrips=None, overlap=None, robin=None):
        S = prob.nstrips if nstrips is None else nstrips
        self.p = _f64(prob.p if S > 1 else np.zeros(1))
        self.q = _f64(prob.q if S > 1 else np.zeros(1))
        self.u0 = _f64(prob.u0)
        self.f_time = _f64(prob.f_time)
        self.f_space = _f64(prob.f_space)
        self.bc_xin = _f64(prob.bc_xin)
        self.bc_v = _f64(prob.bc_v)
        self.desc = _Desc(prob.x0, prob.x1, prob.v0, prob.v1, prob.dt, prob.nx, prob.nv, prob.nt,
                          S, prob.overlap if overlap is None else overlap,
                          int(prob.robin if robin is None else robin), _ptr(self.p), _ptr(self.q),
                          int(getattr(prob, "gauss_seidel", False)), int(getattr(prob, "neumann_v", False)),
                          int(getattr(prob, "periodic_x", False)), int(getattr(prob, "scheme", 0)))
        self.prob = _Problem(_ptr(self.u0), int(self.f_time.shape[0]), _ptr(self.f_time),
                             _ptr(self.f_space), _ptr(self.bc_xin), _ptr(self.bc_v))


def _check(rc):
    if rc != 0:
        raise OracleError({-1: "invalid descriptor", -2: "CFL > 1", -3: "out of memory"}.get(rc, rc))


def trace_shape(prob):
    return (max(prob.nstrips - 1, 0), 2, prob.nt, prob.nx + 1)


def band_shape(prob):
    return (max(prob.nstrips - 1, 0), 2, prob.nt, prob.overlap + 1, prob.nx + 1)


def validate(prob) -> int:
    m = _Marshalled(prob)
    return _load().kfo_validate(ctypes.byref(m.desc))


def strip_layout(prob):
    m = _Marshalled(prob)
    lo = np.zeros(prob.nstrips, np.int32)
    hi = np.zeros(prob.nstrips, np.int32)
    _check(_load().kfo_strip_layout(ctypes.byref(m.desc), lo.ctypes.data_as(_ip), hi.ctypes.data_as(_ip)))
    return lo, hi


def swr_iteration(prob, lam_in: Optional[np.ndarray] = None):
    """One parallel SWR iteration (Section 6.3, SWR1-SWR4 in the Remark's Jacobi form).

    Returns (lam_out, bands, u_T)."""
    m = _Marshalled(prob)
    lam_in = np.zeros(trace_shape(prob)) if lam_in is None else _f64(lam_in)
    lam_out = np.zeros(trace_shape(prob))
    bands = np.zeros(band_shape(prob))
    u_T = np.zeros((prob.nv + 1, prob.nx + 1))
    _check(_load().kfo_swr_iteration(ctypes.byref(m.desc), ctypes.byref(m.prob), _ptr(lam_in),
                                     _ptr(lam_out), _ptr(bands), _ptr(u_T)))
    return lam_out, bands, u_T


def interface_norms(prob, bands, lam_new=None, lam_old=None):
    """(e_mis, e_chg, j_l2) of one iterate (criterion "error" of Section 6.3)."""
    m = _Marshalled(prob)
    out = (ctypes.c_double(), ctypes.c_double(), ctypes.c_double())
    _check(_load().kfo_interface_norms(ctypes.byref(m.desc), _ptr(_f64(bands)), _ptr(_f64(lam_new)),
                                       _ptr(_f64(lam_old)), *[ctypes.byref(o) for o in out]))
    return tuple(o.value for o in out)


def swr_solve(prob, max_iters: int, tol: float = 0.0, tol_kind: int = 0,
              lam0: Optional[np.ndarray] = None):
    """Iterate to tolerance.  Returns dict(lam, iters, hist[(e_mis, e_chg, j_l2)], u_T)."""
    m = _Marshalled(prob)
    if lam0 is None:
        lam0 = prob.lam0
    lam = np.zeros(trace_shape(prob)) if lam0 is None else _f64(lam0).copy()
    hist = np.zeros((max(max_iters, 1), 3))
    u_T = np.zeros((prob.nv + 1, prob.nx + 1))
    iters = ctypes.c_int()
    _check(_load().kfo_swr_solve(ctypes.byref(m.desc), ctypes.byref(m.prob), _ptr(lam), max_iters,
                                 tol, tol_kind, ctypes.byref(iters), _ptr(hist), _ptr(u_T)))
    return {"lam": lam, "iters": iters.value, "hist": hist[: iters.value], "u_T": u_T}


def monolithic(prob, all_levels: bool = False):
    """Single-domain solve of the same scheme.  Returns u_T or (u_T, u_all)."""
    m = _Marshalled(prob, nstrips=1, overlap=0)
    u_T = np.zeros((prob.nv + 1, prob.nx + 1))
    u_all = np.zeros((prob.nt + 1, prob.nv + 1, prob.nx + 1)) if all_levels else None
    _check(_load().kfo_monolithic(ctypes.byref(m.desc), ctypes.byref(m.prob), _ptr(u_T), _ptr(u_all)))
    return (u_T, u_all) if all_levels else u_T


def swr_adjoint(prob, K: int, lam0: Optional[np.ndarray] = None):
    """Discrete adjoint of K parallel SWR iterations (Robin, no overlap): returns
    (J, dJ/dp, dJ/dq), J = dt hx sum (u_j - u_{j+1})^2 on the interface nodes of the
    K-th iterate."""
    m = _Marshalled(prob)
    if lam0 is None:
        lam0 = prob.lam0
    J = ctypes.c_double()
    gp = np.zeros(max(prob.nstrips - 1, 1))
    gq = np.zeros(max(prob.nstrips - 1, 1))
    _check(_load().kfo_swr_adjoint(ctypes.byref(m.desc), ctypes.byref(m.prob), _ptr(_f64(lam0)), K,
                                   ctypes.byref(J), _ptr(gp), _ptr(gq)))
    return J.value, gp[: prob.nstrips - 1], gq[: prob.nstrips - 1]


def thomas(a, b, c, d):
    a, b, c, d = (_f64(z) for z in (a, b, c, d))
    x = np.zeros_like(d)
    _check(_load().kfo_thomas(len(d), _ptr(a), _ptr(b), _ptr(c), _ptr(d), _ptr(x)))
    return x
