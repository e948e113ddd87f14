"""Seeded synthetic problem generators for the SWR sweep of the Kolmogorov equation.

These build the host FP64 arrays that both the CUDA path and the CPU oracle
consume.  The module holds problem data only -- initial densities, forcing
terms, boundary data, random initial interface traces -- and none of the
method's arithmetic (no discretisation, no transmission operator, no solver).

The paper's experiments (Section 6.1) use the error equation (f = 0) on
[0,1] x [-1,1] with a random initial interface value; the larger workloads here
are synthetic stand-ins of the same structure: a Gaussian initial density and a
forcing made of seeded Gaussian bumps.  Every random draw goes through
``numpy.random.default_rng(seed)`` (PCG64) in the order written below.

Array conventions (all C-contiguous float64):
  u0       [nv+1, nx+1]             initial data u0(x_m, v_i), row i = v node
  f_time   [nforce, nt+1]           a_r(t^n)
  f_space  [nforce, nv+1, nx+1]     F_r(x_m, v_i);  f = sum_r a_r(t) F_r(x, v)
  bc_xin   [nt+1, 2, nv+1] or None  inflow data at x0 (index 0) and x1 (index 1)
  bc_v     [nt+1, 2, nx+1] or None  Dirichlet data at v0 (0) and v1 (1)
  lam0     [S-1, 2, nt, nx+1] or None  initial interface traces; [j, 0] is
           lambda_1 (data at the lower strip's top), [j, 1] is lambda_2.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np


@dataclasses.dataclass
class Problem:
    x0: float
    x1: float
    v0: float
    v1: float
    dt: float
    nx: int
    nv: int
    nt: int
    nstrips: int
    overlap: int
    robin: bool
    p: np.ndarray
    q: np.ndarray
    u0: np.ndarray
    f_time: np.ndarray
    f_space: np.ndarray
    bc_xin: Optional[np.ndarray] = None
    bc_v: Optional[np.ndarray] = None
    lam0: Optional[np.ndarray] = None
    name: str = ""
    gauss_seidel: bool = False  # serial SWR1-SWR4 order instead of the parallel form
    neumann_v: bool = False     # homogeneous Neumann at v0, v1 (Section 6.1) instead of Dirichlet data
    periodic_x: bool = False    # periodic in x (Section 6.1): node nx repeats node 0
    scheme: int = 0             # 0: implicit Euler + upwind (finite volumes in v); 1: the Lie
                                # splitting of Section 6.2 with P1 elements in v (model problem)

    @property
    def hx(self) -> float:
        return (self.x1 - self.x0) / self.nx

    @property
    def hv(self) -> float:
        return (self.v1 - self.v0) / self.nv

    @property
    def T(self) -> float:
        return self.nt * self.dt

    def x_nodes(self) -> np.ndarray:
        return self.x0 + np.arange(self.nx + 1) * self.hx

    def v_nodes(self) -> np.ndarray:
        return self.v0 + np.arange(self.nv + 1) * self.hv

    def t_levels(self) -> np.ndarray:
        return np.arange(self.nt + 1) * self.dt

    def replace(self, **kw) -> "Problem":
        """Copy with fields changed; p/q are re-broadcast when the strip count changes."""
        out = dataclasses.replace(self, **kw)
        nif = max(out.nstrips - 1, 0)
        for name in ("p", "q"):
            arr = np.asarray(getattr(out, name), dtype=np.float64).ravel()
            if arr.size != nif:
                fill = float(arr[0]) if arr.size else 1.0
                setattr(out, name, np.full(nif, fill))
        if out.lam0 is not None and out.lam0.shape != (nif, 2, out.nt, out.nx + 1):
            out.lam0 = None
        return out


def _pq(nstrips: int, p, q=None):
    nif = max(nstrips - 1, 0)
    p_arr = np.broadcast_to(np.asarray(p, dtype=np.float64), (nif,)).copy() if nif else np.zeros(0)
    if q is None:
        q_arr = p_arr.copy()
    else:
        q_arr = np.broadcast_to(np.asarray(q, dtype=np.float64), (nif,)).copy() if nif else np.zeros(0)
    return p_arr, q_arr


def manufactured(nx: int = 64, nv: int = 64, nt: int = 20, T: float = 0.1, nstrips: int = 2,
                 overlap: int = 4, robin: bool = False, p: float = 2.0, q: Optional[float] = None) -> Problem:
    """Manufactured solution u = exp(-t) sin(pi x) cos(pi v / 2) on [0,1] x [-1,1].

    Its forcing f = u_t + v u_x - u_vv is exp(-t) [ (pi^2/4 - 1) sin(pi x) cos(pi v/2)
    + pi v cos(pi x) cos(pi v/2) ], and it vanishes on the whole boundary, so all
    boundary data are zero.  One forcing term with a(t) = exp(-t)."""
    x = np.linspace(0.0, 1.0, nx + 1)
    v = -1.0 + np.arange(nv + 1) * (2.0 / nv)
    t = np.arange(nt + 1) * (T / nt)
    X, V = np.meshgrid(x, v, indexing="xy")
    u0 = np.sin(math.pi * X) * np.cos(math.pi * V / 2)
    F = ((math.pi ** 2 / 4 - 1.0) * np.sin(math.pi * X) * np.cos(math.pi * V / 2)
         + math.pi * V * np.cos(math.pi * X) * np.cos(math.pi * V / 2))
    pp, qq = _pq(nstrips, p, q)
    return Problem(0.0, 1.0, -1.0, 1.0, T / nt, nx, nv, nt, nstrips, overlap, robin, pp, qq,
                   np.ascontiguousarray(u0), np.exp(-t)[None, :].copy(), np.ascontiguousarray(F[None]),
                   name=f"manufactured nx={nx} nv={nv} nt={nt}")


def gaussian_bumps(nx: int, nv: int, nt: int, dt: float, nstrips: int, p=4.0, q=None, seed: int = 2,
                   nbumps: int = 16, overlap: int = 0, robin: bool = True,
                   x_range=(0.0, 1.0), v_range=(-4.0, 4.0)) -> Problem:
    """Gaussian initial density plus a forcing of seeded Gaussian bumps, zero boundary data.

    Draw order (rng = default_rng(seed)): amplitudes A ~ U[0,1], widths
    w ~ U[0.02, 0.1], centres x_k ~ U[0.1, 0.9], centres v_k ~ U[-3, 3], each as a
    vector of ``nbumps``.  F(x,v) = sum_k A_k exp(-(x-x_k)^2/(2w_k^2)) exp(-(v-v_k)^2/(2w_k^2));
    a(t) = 1.  u0 = exp(-(x-0.5)^2/(2*0.1^2) - v^2/(2*0.5^2))."""
    rng = np.random.default_rng(seed)
    A = rng.uniform(0.0, 1.0, nbumps)
    w = rng.uniform(0.02, 0.1, nbumps)
    xk = rng.uniform(0.1, 0.9, nbumps)
    vk = rng.uniform(-3.0, 3.0, nbumps)
    x0, x1 = x_range
    v0, v1 = v_range
    x = x0 + np.arange(nx + 1) * ((x1 - x0) / nx)
    v = v0 + np.arange(nv + 1) * ((v1 - v0) / nv)
    F = np.zeros((nv + 1, nx + 1))
    for k in range(nbumps):
        gx = np.exp(-((x - xk[k]) ** 2) / (2 * w[k] ** 2))
        gv = np.exp(-((v - vk[k]) ** 2) / (2 * w[k] ** 2))
        F += A[k] * np.outer(gv, gx)
    gx0 = np.exp(-((x - 0.5) ** 2) / (2 * 0.1 ** 2))
    gv0 = np.exp(-(v ** 2) / (2 * 0.5 ** 2))
    u0 = np.outer(gv0, gx0)
    pp, qq = _pq(nstrips, p, q)
    return Problem(x0, x1, v0, v1, dt, nx, nv, nt, nstrips, overlap, robin, pp, qq,
                   np.ascontiguousarray(u0), np.ones((1, nt + 1)), F[None].copy(),
                   name=f"gaussian bumps nx={nx} nv={nv} nt={nt} S={nstrips} seed={seed}")


def error_equation(nx: int, nv: int, nt: int, dt: float, nstrips: int, overlap: int, robin: bool,
                   p=2.0, q=None, seed: int = 0, x_range=(0.0, 1.0), v_range=(-1.0, 1.0)) -> Problem:
    """The error equation of Section 6.1: f = 0, u0 = 0, zero boundary data, and a
    random initial interface value lambda^0 ~ U[-1, 1] (rng = default_rng(seed),
    one draw of shape [S-1, 2, nt, nx+1]), so that every frequency is present."""
    rng = np.random.default_rng(seed)
    pp, qq = _pq(nstrips, p, q)
    lam0 = rng.uniform(-1.0, 1.0, (max(nstrips - 1, 0), 2, nt, nx + 1))
    return Problem(x_range[0], x_range[1], v_range[0], v_range[1], dt, nx, nv, nt, nstrips, overlap,
                   robin, pp, qq, np.zeros((nv + 1, nx + 1)), np.zeros((1, nt + 1)),
                   np.zeros((1, nv + 1, nx + 1)), lam0=lam0,
                   name=f"error equation nx={nx} nv={nv} nt={nt} S={nstrips} ov={overlap} seed={seed}")


def random_data(nx: int, nv: int, nt: int, dt: float, nstrips: int, overlap: int, robin: bool,
                p=2.0, q=None, seed: int = 0, nforce: int = 2, v_range=(-1.0, 1.0),
                constant_in_time: bool = False, boundary_data: bool = True) -> Problem:
    """Every input drawn at random (rng = default_rng(seed), draw order: u0, f_time,
    f_space, bc_xin, bc_v, lam0; all U[-1, 1]).  Exercises every data path: both
    inflow sides, both v boundaries, forcing terms and nonzero traces.  With
    ``constant_in_time`` every a_r(t^n) equals its value at n = 1; without
    ``boundary_data`` the inflow and v-boundary data are zero (passed as None),
    after the same draws."""
    rng = np.random.default_rng(seed)
    u0 = rng.uniform(-1, 1, (nv + 1, nx + 1))
    f_time = rng.uniform(-1, 1, (nforce, nt + 1))
    if constant_in_time:
        f_time[:, 1:] = f_time[:, 1:2]
    f_space = rng.uniform(-1, 1, (nforce, nv + 1, nx + 1))
    bc_xin = rng.uniform(-1, 1, (nt + 1, 2, nv + 1))
    bc_v = rng.uniform(-1, 1, (nt + 1, 2, nx + 1))
    lam0 = rng.uniform(-1, 1, (max(nstrips - 1, 0), 2, nt, nx + 1))
    if not boundary_data:
        bc_xin = bc_v = None
    pp, qq = _pq(nstrips, p, q)
    return Problem(0.0, 1.0, v_range[0], v_range[1], dt, nx, nv, nt, nstrips, overlap, robin, pp, qq,
                   u0, f_time, f_space, bc_xin, bc_v, lam0,
                   name=f"random data nx={nx} nv={nv} nt={nt} S={nstrips} ov={overlap} seed={seed}")


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------

def small_dirichlet() -> Problem:
    """x in [0,1], v in [-1,1], 64 x 64 cells, 2 strips split at v = 0, Dirichlet
    transmission with a 4-cell overlap, T = 0.1, dt = 0.005 (20 steps), manufactured
    solution; iterate until the interface change is below 1e-10 or 50 iterations."""
    return manufactured(64, 64, 20, 0.1, nstrips=2, overlap=4, robin=False)


def small_robin() -> Problem:
    """As ``small_dirichlet`` but non-overlapping with Robin transmission p = q = 2."""
    return manufactured(64, 64, 20, 0.1, nstrips=2, overlap=0, robin=True, p=2.0)


def at_scale(seed: int = 2) -> Problem:
    """x in [0,1], v in [-4,4], 2048 x 4096 cells, 8 equal v-strips, Robin p = 4 without
    overlap, dt = 1e-4 and 2000 steps (CFL 0.8192), 16 seeded Gaussian bumps; 30 iterations."""
    return gaussian_bumps(2048, 4096, 2000, 1e-4, nstrips=8, p=4.0, seed=seed)


def mixed_precision_workload(seed: int = 4) -> Problem:
    """x in [0,1], v in [-4,4], 4096 x 8192 cells, 16 Robin strips p = 4, dt = 5e-5,
    4000 steps, seeded Gaussian bumps."""
    return gaussian_bumps(4096, 8192, 4000, 5e-5, nstrips=16, p=4.0, seed=seed)


def adjoint_workload(seed: int = 5) -> Problem:
    """512 x 1024 cells, 8 Robin strips (7 interface parameters, initial p = 4),
    dt = 4e-4, 500 steps, seeded Gaussian bumps."""
    return gaussian_bumps(512, 1024, 500, 4e-4, nstrips=8, p=4.0, seed=seed)


def model_error_equation(j: int = 0, overlap: int = 3, robin: bool = True, p=4.23, q=None, seed: int = 7,
                         T: float = 2.0, nstrips: int = 2) -> Problem:
    """Error equation of the model problem of Section 6.1 in the setting of Section 6.4 and
    Table 1: x in [0,1] periodic, v in [-1,1] with zero flux, f = 0, u0 = 0, T = 2,
    hx = hv = dt = 0.01 * 2^-j (so nx = 100 * 2^j, nv = nt = 200 * 2^j), strips split
    at v = 0, random initial data lambda_1^0 ~ U[-1,1] (default_rng(seed), one draw of
    shape [S-1][nt][nx+1]) and lambda_2^0 = 0."""
    n = 100 * 2 ** j
    h = 1.0 / n
    nx, nv, nt = n, 2 * n, int(round(T / h))
    rng = np.random.default_rng(seed)
    lam0 = np.zeros((nstrips - 1, 2, nt, nx + 1))
    lam0[:, 0] = rng.uniform(-1, 1, (nstrips - 1, nt, nx + 1))
    pp, qq = _pq(nstrips, p, q)
    return Problem(0.0, 1.0, -1.0, 1.0, h, nx, nv, nt, nstrips, overlap, robin, pp, qq,
                   np.zeros((nv + 1, nx + 1)), np.zeros((1, nt + 1)), np.zeros((1, nv + 1, nx + 1)),
                   None, None, lam0, neumann_v=True, periodic_x=True,
                   name=f"model error equation j={j} ov={overlap} {'Robin' if robin else 'Dirichlet'}")


def batch_instances(count: int = 256, seed_base: int = 3000, v_range=(-4.0, 4.0)) -> List[Problem]:
    """Uneven instances for the batched form.  Instance i uses rng = default_rng(seed_base + i)
    and draws, in order: nx ~ U{128..1024}; S ~ U{2,4,8,16}; cells per strip
    ~ U{ceil(256/S)..floor(2048/S)} (so nv = S * that); log p ~ U[log 0.5, log 16];
    nt ~ U{200..1000}; then a bump seed ~ U{0..2^31-1}.  dt = 0.8 hx / 4 (CFL 0.8)."""
    out = []
    for k in range(count):
        rng = np.random.default_rng(seed_base + k)
        nx = int(rng.integers(128, 1025))
        S = int(rng.choice([2, 4, 8, 16]))
        w = int(rng.integers(math.ceil(256 / S), 2048 // S + 1))
        p = float(np.exp(rng.uniform(math.log(0.5), math.log(16.0))))
        nt = int(rng.integers(200, 1001))
        bseed = int(rng.integers(0, 2 ** 31 - 1))
        hx = 1.0 / nx
        dt = 0.8 * hx / max(abs(v_range[0]), abs(v_range[1]))
        prob = gaussian_bumps(nx, S * w, nt, dt, nstrips=S, p=p, seed=bseed, v_range=v_range)
        prob.name = f"batch[{k}] nx={nx} nv={S * w} S={S} nt={nt} p={p:.3f}"
        out.append(prob)
    return out
