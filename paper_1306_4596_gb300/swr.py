"""Python binding of the C ABI in ``include/kfp_swr.h`` (argument marshalling only).

The functions ``kfp_swr_create`` ... ``kfp_swr_destroy`` carry the C names and
arguments one to one; every step of the method runs in the CUDA library.  PyTorch
is used for device memory and for the stream handle only.  There is no CPU
fallback: if ``libkfp_swr.so`` cannot be built or loaded, every call raises.

``SWR`` is a small convenience wrapper that takes an ``inputs.Problem``.
"""
from __future__ import annotations

import ctypes
import threading
from typing import Optional

import numpy as np

from . import build as _build

KFP_OK, KFP_EINVAL, KFP_ECFL, KFP_ENOMEM, KFP_ECUDA, KFP_ENOTCONV, KFP_ENUMERIC, KFP_ETIMEOUT, KFP_ENOTSUP = range(9)
STATUS_NAMES = {0: "KFP_OK", 1: "KFP_EINVAL", 2: "KFP_ECFL", 3: "KFP_ENOMEM", 4: "KFP_ECUDA",
                5: "KFP_ENOTCONV", 6: "KFP_ENUMERIC", 7: "KFP_ETIMEOUT", 8: "KFP_ENOTSUP"}
KFP_DIRICHLET, KFP_ROBIN = 0, 1
KFP_F64, KFP_F32, KFP_MIXED = 0, 1, 2
PRECISIONS = {"f64": KFP_F64, "f32": KFP_F32, "mixed": KFP_MIXED}
KFP_FLAG_NO_GRAPH, KFP_FLAG_PROFILE, KFP_FLAG_GENERIC, KFP_FLAG_GAUSS_SEIDEL = 1, 2, 4, 8
KFP_FLAG_NEUMANN_V, KFP_FLAG_PERIODIC_X, KFP_FLAG_SPLIT_SCHEME, KFP_FLAG_PERSISTENT = 16, 32, 64, 128
KFP_FLAG_PER_PASS = 256
KFP_FLAG_SHAPE_SHIFT = 9
KFP_FLAG_DEPTH_SHIFT = 11
TILE_SHAPES = 3
MAX_DEPTH = 8


def KFP_FLAG_SHAPE(n: int) -> int:
    """Flag fixing the tile shape n (0..2) of the TMA-fed sweep."""
    return (n + 1) << KFP_FLAG_SHAPE_SHIFT


def KFP_FLAG_DEPTH(n: int) -> int:
    """Flag fixing the number n (1..8) of consecutive iterates swept together (1: none)."""
    return n << KFP_FLAG_DEPTH_SHIFT


def problem_flags(prob) -> int:
    """Flags that a problem's own definition sets: iteration order and boundary conditions."""
    return ((KFP_FLAG_GAUSS_SEIDEL if getattr(prob, "gauss_seidel", False) else 0)
            | (KFP_FLAG_NEUMANN_V if getattr(prob, "neumann_v", False) else 0)
            | (KFP_FLAG_PERIODIC_X if getattr(prob, "periodic_x", False) else 0)
            | (KFP_FLAG_SPLIT_SCHEME if getattr(prob, "scheme", 0) == 1 else 0))

EXPORTED = ("kfp_swr_create", "kfp_swr_sweep", "kfp_swr_traces", "kfp_swr_set_traces", "kfp_swr_error",
            "kfp_swr_bands", "kfp_swr_solution", "kfp_swr_stats", "kfp_swr_destroy",
            "kfp_swr_last_error", "kfp_swr_create_error", "kfp_iface_norms_noalloc", "kfp_swr_counters",
            "kfp_batch_create", "kfp_batch_configure", "kfp_batch_sweep", "kfp_batch_instance", "kfp_batch_stats",
            "kfp_batch_destroy", "kfp_batch_last_error", "kfp_swr_gradient", "kfp_swr_set_robin",
            "kfp_selftest_bounded_wait", "kfp_swr_selftest_stall", "kfp_probe_fp64_rate")
KFP_NOALLOC_MAX_INTERFACES = 64

_dp = ctypes.POINTER(ctypes.c_double)


class kfp_swr_desc(ctypes.Structure):
    _fields_ = [
        ("x0", ctypes.c_double), ("x1", ctypes.c_double), ("v0", ctypes.c_double), ("v1", ctypes.c_double),
        ("dt", ctypes.c_double), ("nx", ctypes.c_int), ("nv", ctypes.c_int), ("nt", ctypes.c_int),
        ("nstrips", ctypes.c_int), ("overlap_cells", ctypes.c_int), ("tc", ctypes.c_int),
        ("p", ctypes.c_void_p), ("q", ctypes.c_void_p), ("prec", ctypes.c_int), ("flags", ctypes.c_uint),
    ]


class kfp_swr_problem(ctypes.Structure):
    _fields_ = [
        ("on_device", ctypes.c_int), ("u0", ctypes.c_void_p), ("nforce", ctypes.c_int),
        ("f_time", ctypes.c_void_p), ("f_space", ctypes.c_void_p), ("bc_xin", ctypes.c_void_p),
        ("bc_v", ctypes.c_void_p), ("lambda0", ctypes.c_void_p),
    ]


class KfpError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None
_lock = threading.Lock()


def load(rebuild: bool = False):
    """Build (if stale) and load ``libkfp_swr.so``; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is None or rebuild:
            path = _build.build(force=rebuild)
            lib = ctypes.CDLL(path)
            vp, ip, i = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int
            llp = ctypes.POINTER(ctypes.c_longlong)
            lib.kfp_swr_create.argtypes = [ctypes.POINTER(kfp_swr_desc), ctypes.POINTER(kfp_swr_problem), vp,
                                           ctypes.POINTER(vp)]
            lib.kfp_swr_sweep.argtypes = [vp, i, ctypes.c_double, i, ip]
            lib.kfp_swr_traces.argtypes = [vp, i, i, vp, i]
            lib.kfp_swr_set_traces.argtypes = [vp, vp, i]
            lib.kfp_swr_error.argtypes = [vp, _dp, _dp, _dp, _dp, i]
            lib.kfp_swr_bands.argtypes = [vp, i, i, vp, i]
            lib.kfp_swr_solution.argtypes = [vp, vp, i]
            lib.kfp_swr_stats.argtypes = [vp, llp, llp, ip, _dp, _dp, _dp]
            lib.kfp_swr_pipeline_stats.argtypes = [vp, ip, llp, llp, llp, _dp]
            lib.kfp_swr_gradient.argtypes = [vp, i, vp, i, _dp, _dp, _dp]
            lib.kfp_swr_gradient.restype = ctypes.c_int
            lib.kfp_swr_set_robin.argtypes = [vp, vp, vp]
            lib.kfp_swr_set_robin.restype = ctypes.c_int
            lib.kfp_swr_counters.argtypes = [vp, llp, llp, _dp]
            lib.kfp_swr_counters.restype = ctypes.c_int
            lib.kfp_batch_create.argtypes = [ctypes.POINTER(kfp_swr_desc), ctypes.POINTER(kfp_swr_problem), i, vp,
                                             ctypes.POINTER(vp)]
            lib.kfp_batch_configure.argtypes = [vp, i, i, i]
            lib.kfp_batch_sweep.argtypes = [vp, i, ctypes.c_double, i, ip]
            lib.kfp_batch_instance.argtypes = [vp, i, ctypes.POINTER(vp)]
            lib.kfp_batch_stats.argtypes = [vp, llp, llp, _dp, _dp]
            lib.kfp_batch_destroy.argtypes = [vp]
            lib.kfp_batch_destroy.restype = None
            lib.kfp_batch_last_error.argtypes = [vp]
            lib.kfp_batch_last_error.restype = ctypes.c_char_p
            for name in ("kfp_batch_create", "kfp_batch_configure", "kfp_batch_sweep", "kfp_batch_instance",
                         "kfp_batch_stats"):
                getattr(lib, name).restype = ctypes.c_int
            lib.kfp_swr_destroy.argtypes = [vp]
            lib.kfp_swr_destroy.restype = None
            lib.kfp_swr_last_error.argtypes = [vp]
            lib.kfp_swr_last_error.restype = ctypes.c_char_p
            lib.kfp_iface_norms_noalloc.argtypes = [vp, i, i, i, i, i, ctypes.c_double, ctypes.c_double, vp, vp]
            lib.kfp_iface_norms_noalloc.restype = ctypes.c_int
            lib.kfp_probe_fp64_rate.argtypes = [i, i, i, _dp, _dp, vp]
            lib.kfp_probe_fp64_rate.restype = ctypes.c_int
            lib.kfp_swr_selftest_stall.argtypes = [vp, i, ctypes.c_double]
            lib.kfp_swr_selftest_stall.restype = ctypes.c_int
            lib.kfp_swr_create_error.argtypes = []
            lib.kfp_swr_create_error.restype = ctypes.c_char_p
            for name in ("kfp_swr_create", "kfp_swr_sweep", "kfp_swr_traces", "kfp_swr_set_traces",
                         "kfp_swr_error", "kfp_swr_bands", "kfp_swr_solution", "kfp_swr_stats"):
                getattr(lib, name).restype = ctypes.c_int
            _lib = lib
    return _lib


def _check(h, status: int, allow=()):
    if status != KFP_OK and status not in allow:
        msg = _lib.kfp_swr_last_error(h).decode() if h else _lib.kfp_swr_create_error().decode()
        raise KfpError(status, msg)
    return status


# ---------------------------------------------------------------------------
# C entry points, same names and arguments
# ---------------------------------------------------------------------------

def kfp_swr_create(desc: kfp_swr_desc, prob: kfp_swr_problem, cuda_stream: int = 0) -> int:
    lib = load()
    out = ctypes.c_void_p()
    st = lib.kfp_swr_create(ctypes.byref(desc), ctypes.byref(prob), ctypes.c_void_p(cuda_stream), ctypes.byref(out))
    _check(None, st)
    return out.value


def kfp_swr_sweep(h: int, max_iters: int, tol: float = 0.0, tol_kind: int = 0, allow_notconv: bool = False) -> int:
    done = ctypes.c_int()
    st = load().kfp_swr_sweep(h, max_iters, tol, tol_kind, ctypes.byref(done))
    _check(h, st, allow=(KFP_ENOTCONV,) if allow_notconv else ())
    return done.value


def kfp_swr_traces(h: int, iface: int, side: int, dst_ptr: int, dst_on_device: int) -> None:
    _check(h, load().kfp_swr_traces(h, iface, side, dst_ptr, dst_on_device))


def kfp_swr_set_traces(h: int, src_ptr: int, src_on_device: int) -> None:
    _check(h, load().kfp_swr_set_traces(h, src_ptr, src_on_device))


def kfp_swr_error(h: int, hist_cap: int = 0):
    e = (ctypes.c_double(), ctypes.c_double(), ctypes.c_double())
    hist = np.zeros((max(hist_cap, 1), 3))
    _check(h, load().kfp_swr_error(h, *[ctypes.byref(x) for x in e],
                                   hist.ctypes.data_as(_dp) if hist_cap > 0 else None, hist_cap))
    return e[0].value, e[1].value, e[2].value, hist[:hist_cap]


def kfp_swr_bands(h: int, iface: int, side: int, dst_ptr: int, dst_on_device: int) -> None:
    _check(h, load().kfp_swr_bands(h, iface, side, dst_ptr, dst_on_device))


def kfp_swr_solution(h: int, dst_ptr: int, dst_on_device: int) -> None:
    _check(h, load().kfp_swr_solution(h, dst_ptr, dst_on_device))


def kfp_swr_stats(h: int) -> dict:
    it, cells = ctypes.c_longlong(), ctypes.c_longlong()
    launches = ctypes.c_int()
    t = (ctypes.c_double(), ctypes.c_double(), ctypes.c_double())
    _check(h, load().kfp_swr_stats(h, ctypes.byref(it), ctypes.byref(cells), ctypes.byref(launches),
                                   *[ctypes.byref(x) for x in t]))
    return {"iterations": it.value, "cell_updates_per_iter": cells.value, "launches_per_iter": launches.value,
            "sweep_ms": t[0].value, "exchange_ms": t[1].value, "error_ms": t[2].value}


def kfp_swr_pipeline_stats(h: int) -> dict:
    depth = ctypes.c_int()
    kernels, launches, cells = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
    ms = ctypes.c_double()
    _check(h, load().kfp_swr_pipeline_stats(h, ctypes.byref(depth), ctypes.byref(kernels), ctypes.byref(launches),
                                            ctypes.byref(cells), ctypes.byref(ms)))
    return {"depth": depth.value, "kernel_launches": kernels.value, "stream_launches": launches.value,
            "stream_cell_updates": cells.value, "stream_ms": ms.value}


def kfp_swr_counters(h: int) -> dict:
    a, b = ctypes.c_longlong(), ctypes.c_longlong()
    t = ctypes.c_double()
    _check(h, load().kfp_swr_counters(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(t)))
    return {"fp64_iterations": a.value, "fp32_iterations": b.value, "fp32_sweep_ms": t.value}


def kfp_swr_gradient(h: int, K: int, lam0_ptr=None, lam0_on_device: int = 0, nif: int = 1):
    """(J, dJ/dp, dJ/dq) after K iterations from lambda^0 (discrete adjoint)."""
    J = ctypes.c_double()
    gp = np.zeros(max(nif, 1))
    gq = np.zeros(max(nif, 1))
    _check(h, load().kfp_swr_gradient(h, K, lam0_ptr, lam0_on_device, ctypes.byref(J), gp.ctypes.data_as(_dp),
                                      gq.ctypes.data_as(_dp)))
    return J.value, gp[:nif], gq[:nif]


def kfp_swr_set_robin(h: int, p, q=None) -> None:
    p = np.ascontiguousarray(p, dtype=np.float64)
    q = None if q is None else np.ascontiguousarray(q, dtype=np.float64)
    _check(h, load().kfp_swr_set_robin(h, p.ctypes.data, None if q is None else q.ctypes.data))


def kfp_swr_destroy(h: int) -> None:
    if h:
        load().kfp_swr_destroy(h)


def kfp_iface_norms_noalloc(bands_ptr: int, nif: int, nt: int, overlap_cells: int, nx: int, dt: float, hx: float,
                            out_ptr: int, cuda_stream: int = 0, periodic_x: bool = False) -> None:
    """Interface norms from device-resident overlap values, with no allocation (see the header)."""
    st = load().kfp_iface_norms_noalloc(bands_ptr, nif, nt, overlap_cells, nx, int(bool(periodic_x)), dt, hx,
                                        out_ptr, cuda_stream)
    if st != KFP_OK:
        if st == KFP_EINVAL and nif > KFP_NOALLOC_MAX_INTERFACES:
            msg = f"nif = {nif} exceeds KFP_NOALLOC_MAX_INTERFACES = {KFP_NOALLOC_MAX_INTERFACES}"
        elif st == KFP_EINVAL:
            msg = "NULL pointer, non-positive size, or periodic x with nx < 2"
        else:
            msg = "device set-up or kernel launch failed"
        raise KfpError(st, f"kfp_iface_norms_noalloc: {msg}")


def kfp_selftest_bounded_wait(limit: int = 1 << 16, cuda_stream: int = 0) -> int:
    """Run the bounded-wait check (see the header); returns the status, KFP_ETIMEOUT
    when the wait gave up as designed."""
    lib = load()
    lib.kfp_selftest_bounded_wait.argtypes = [ctypes.c_uint, ctypes.c_void_p]
    return int(lib.kfp_selftest_bounded_wait(limit, cuda_stream))


def kfp_swr_selftest_stall(h: int, unit: int, limit_s: float) -> int:
    """Run the sweep passes once with one unit never reporting completion (see the
    header); returns the status, KFP_ETIMEOUT when the waits gave up as designed."""
    return int(load().kfp_swr_selftest_stall(h, unit, limit_s))


def kfp_probe_fp64_rate(chains: int = 8, warps_per_sm: int = 16, steps: int = 20000, cuda_stream: int = 0):
    """(DFMA operations per second, SM MHz during the run) of the current device (see the header)."""
    rate, mhz = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = load().kfp_probe_fp64_rate(chains, warps_per_sm, steps, ctypes.byref(rate), ctypes.byref(mhz), cuda_stream)
    if st != KFP_OK:
        raise KfpError(st, "kfp_probe_fp64_rate failed")
    return rate.value, mhz.value


def kfp_swr_last_error(h: int) -> str:
    return load().kfp_swr_last_error(h).decode()


# ---------------------------------------------------------------------------
# Convenience wrapper
# ---------------------------------------------------------------------------

def cell_updates_per_iteration(prob) -> int:
    """Strip nodes advanced per iteration: (nx+1) * sum_s (hi_s - lo_s + 1) * nt."""
    S, w, ov = prob.nstrips, prob.nv // prob.nstrips, (prob.overlap if prob.nstrips > 1 else 0)
    nodes = 0
    for s in range(S):
        lo = 0 if s == 0 else s * w - ov // 2
        hi = prob.nv if s == S - 1 else (s + 1) * w - ov // 2 + ov
        nodes += hi - lo + 1
    return (prob.nx + 1) * nodes * prob.nt


def _marshal(prob, precision: str, flags: int, inputs_on: str, keep: list):
    """Build (kfp_swr_desc, kfp_swr_problem) for a Problem; buffers are appended to keep."""
    import torch

    on_dev = inputs_on == "device"

    def put(a):
        if a is None:
            return None
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
        t = t.to("cuda") if on_dev else t.pin_memory()
        keep.append(t)
        return t.data_ptr()

    S = prob.nstrips
    flags |= problem_flags(prob)
    p = np.ascontiguousarray(prob.p, dtype=np.float64) if S > 1 else None
    q = np.ascontiguousarray(prob.q, dtype=np.float64) if S > 1 else None
    keep.extend([p, q])
    desc = kfp_swr_desc(prob.x0, prob.x1, prob.v0, prob.v1, prob.dt, prob.nx, prob.nv, prob.nt, S, prob.overlap,
                        KFP_ROBIN if prob.robin else KFP_DIRICHLET, p.ctypes.data if p is not None else None,
                        q.ctypes.data if q is not None else None, PRECISIONS[precision], flags)
    cdata = kfp_swr_problem(1 if on_dev else 0, put(prob.u0), int(prob.f_time.shape[0]), put(prob.f_time),
                            put(prob.f_space), put(prob.bc_xin), put(prob.bc_v), put(prob.lam0))
    return desc, cdata


class Batch:
    """Independent problems swept together (one launch per time step for all)."""

    def __init__(self, probs, precision: str = "f64", stream=None, inputs_on: str = "device", graph: bool = True,
                 profile: bool = False):
        import torch

        self.probs = list(probs)
        self.stream = torch.cuda.current_stream() if stream is None else stream
        keep = []
        flags = (0 if graph else KFP_FLAG_NO_GRAPH) | (KFP_FLAG_PROFILE if profile else 0)
        pairs = [_marshal(p, precision, flags, inputs_on, keep) for p in self.probs]
        descs = (kfp_swr_desc * len(pairs))(*[d for d, _ in pairs])
        cdat = (kfp_swr_problem * len(pairs))(*[c for _, c in pairs])
        if inputs_on == "device":
            torch.cuda.current_stream().synchronize()
        lib = load()
        out = ctypes.c_void_p()
        st = lib.kfp_batch_create(descs, cdat, len(pairs), ctypes.c_void_p(int(self.stream.cuda_stream)),
                                  ctypes.byref(out))
        if st != KFP_OK:
            raise KfpError(st, lib.kfp_batch_last_error(None).decode())
        self.b = out.value
        self._handles = {}

    def _check(self, st, allow=()):
        if st != KFP_OK and st not in allow:
            raise KfpError(st, load().kfp_batch_last_error(self.b).decode())
        return st

    def configure(self, blocks_per_sm: int = 0, unit_order: int = 0, tile_shape: int = 1) -> None:
        self._check(load().kfp_batch_configure(self.b, blocks_per_sm, unit_order, tile_shape))

    def sweep(self, max_iters: int, tol: float = 0.0, tol_kind: int = 0, allow_notconv: bool = True) -> int:
        done = ctypes.c_int()
        self._check(load().kfp_batch_sweep(self.b, max_iters, tol, tol_kind, ctypes.byref(done)),
                    allow=(KFP_ENOTCONV,) if allow_notconv else ())
        return done.value

    def handle(self, index: int) -> int:
        if index not in self._handles:
            h = ctypes.c_void_p()
            self._check(load().kfp_batch_instance(self.b, index, ctypes.byref(h)))
            self._handles[index] = h.value
        return self._handles[index]

    def view(self, index: int) -> "SWR":
        """An SWR-like read-only view of problem `index` (results only)."""
        v = SWR.__new__(SWR)
        v.prob = self.probs[index]
        v.h = self.handle(index)
        v._owned = False
        return v

    def stats(self) -> dict:
        it, cells = ctypes.c_longlong(), ctypes.c_longlong()
        a, b = ctypes.c_double(), ctypes.c_double()
        self._check(load().kfp_batch_stats(self.b, ctypes.byref(it), ctypes.byref(cells), ctypes.byref(a),
                                           ctypes.byref(b)))
        return {"iterations": it.value, "cell_updates_per_iter": cells.value, "sweep_ms": a.value,
                "reduce_ms": b.value}

    def close(self) -> None:
        if getattr(self, "b", None):
            load().kfp_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class SWR:
    """One problem resident on the current CUDA device.

    ``inputs_on`` = "device": the problem arrays are first copied into torch CUDA
    tensors and handed over as device pointers; "host": host (pinned) pointers are
    handed over and the library copies them in.  ``persistent``, ``tile_shape`` and
    ``depth`` fix how the sweep is launched (KFP_FLAG_PERSISTENT / KFP_FLAG_PER_PASS,
    KFP_FLAG_SHAPE, KFP_FLAG_DEPTH); None lets the library choose.  Every choice gives
    the same bits."""

    def __init__(self, prob, precision: str = "f64", stream=None, inputs_on: str = "device",
                 graph: bool = True, profile: bool = False, generic: bool = False, persistent: Optional[bool] = None,
                 tile_shape: Optional[int] = None, depth: Optional[int] = None):
        import torch

        self.prob = prob
        self._torch = torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        S = prob.nstrips
        self._keep = []
        on_dev = inputs_on == "device"

        def put(a):
            if a is None:
                return None
            t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
            if on_dev:
                t = t.to("cuda", non_blocking=False)
            else:
                t = t.pin_memory()
            self._keep.append(t)
            return t.data_ptr()

        self._p = np.ascontiguousarray(prob.p, dtype=np.float64) if S > 1 else None
        self._q = np.ascontiguousarray(prob.q, dtype=np.float64) if S > 1 else None
        flags = ((0 if graph else KFP_FLAG_NO_GRAPH) | (KFP_FLAG_PROFILE if profile else 0)
                 | (KFP_FLAG_GENERIC if generic else 0)
                 | {None: 0, True: KFP_FLAG_PERSISTENT, False: KFP_FLAG_PER_PASS}[persistent]
                 | (0 if tile_shape is None else KFP_FLAG_SHAPE(tile_shape))
                 | (0 if depth is None else KFP_FLAG_DEPTH(depth))
                 | problem_flags(prob))
        self.desc = kfp_swr_desc(prob.x0, prob.x1, prob.v0, prob.v1, prob.dt, prob.nx, prob.nv, prob.nt, S,
                                 prob.overlap, KFP_ROBIN if prob.robin else KFP_DIRICHLET,
                                 self._p.ctypes.data if self._p is not None else None,
                                 self._q.ctypes.data if self._q is not None else None,
                                 PRECISIONS[precision], flags)
        nforce = int(prob.f_time.shape[0])
        self.cdata = kfp_swr_problem(1 if on_dev else 0, put(prob.u0), nforce, put(prob.f_time),
                                     put(prob.f_space), put(prob.bc_xin), put(prob.bc_v), put(prob.lam0))
        if on_dev:
            torch.cuda.current_stream().synchronize()
        self.h = kfp_swr_create(self.desc, self.cdata, int(stream.cuda_stream))
        self._keep.clear()  # inputs were copied

    # -- iteration ---------------------------------------------------------------
    def sweep(self, max_iters: int, tol: float = 0.0, tol_kind: int = 0, allow_notconv: bool = True) -> int:
        return kfp_swr_sweep(self.h, max_iters, tol, tol_kind, allow_notconv=allow_notconv)

    # -- results -----------------------------------------------------------------
    def traces(self) -> np.ndarray:
        p = self.prob
        out = np.zeros((max(p.nstrips - 1, 0), 2, p.nt, p.nx + 1))
        for j in range(p.nstrips - 1):
            for side in range(2):
                kfp_swr_traces(self.h, j, side, out[j, side].ctypes.data, 0)
        return out

    def set_traces(self, lam: np.ndarray) -> None:
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        kfp_swr_set_traces(self.h, lam.ctypes.data, 0)

    def bands(self) -> np.ndarray:
        p = self.prob
        out = np.zeros((max(p.nstrips - 1, 0), 2, p.nt, p.overlap + 1, p.nx + 1))
        for j in range(p.nstrips - 1):
            for side in range(2):
                kfp_swr_bands(self.h, j, side, out[j, side].ctypes.data, 0)
        return out

    def solution(self) -> np.ndarray:
        out = np.zeros((self.prob.nv + 1, self.prob.nx + 1))
        kfp_swr_solution(self.h, out.ctypes.data, 0)
        return out

    def solution_device(self):
        out = self._torch.empty((self.prob.nv + 1, self.prob.nx + 1), dtype=self._torch.float64, device="cuda")
        kfp_swr_solution(self.h, out.data_ptr(), 1)
        return out

    def error(self):
        """(e_mis, e_chg, j_l2, history[iterations, 3])."""
        st = kfp_swr_stats(self.h)
        return kfp_swr_error(self.h, int(st["iterations"]))

    def stats(self) -> dict:
        return kfp_swr_stats(self.h)

    def pipeline_stats(self) -> dict:
        return kfp_swr_pipeline_stats(self.h)

    def counters(self) -> dict:
        return kfp_swr_counters(self.h)

    def gradient(self, K: int, lam0: Optional[np.ndarray] = None):
        """(J, dJ/dp, dJ/dq): J = dt hx sum (u_j - u_{j+1})^2 on the interface nodes after
        K iterations from lam0 (None = 0)."""
        lam = None if lam0 is None else np.ascontiguousarray(lam0, dtype=np.float64)
        return kfp_swr_gradient(self.h, K, None if lam is None else lam.ctypes.data, 0, self.prob.nstrips - 1)

    def set_robin(self, p, q=None) -> None:
        kfp_swr_set_robin(self.h, p, q)
        self.prob = self.prob.replace()
        self.prob.p = np.array(p, dtype=np.float64)
        self.prob.q = np.array(p if q is None else q, dtype=np.float64)

    def close(self) -> None:
        if getattr(self, "h", None) and getattr(self, "_owned", True):
            kfp_swr_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
