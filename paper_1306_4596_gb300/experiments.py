"""Experiments of Section 6 run on the CUDA path.

* ``table1``: iteration counts of CSWR, OSWR(p) (p = q = 4.23) and OSWR(p,q) (p = 11,
  q = 2.5) to bring the interface mismatch e_mis below 1e-6, with an overlap of three
  cells and without overlap, under the dyadic refinement hx = hv = dt = 0.01 * 2^-j
  (Section 6.5, Table 1).
* ``p_scan``: iterations to e_mis < 1e-6 and e_mis after 15 iterations as functions
  of the one-sided Robin parameter p (Section 6.4.1, Figure 1).
* ``pq_scan``: the same over a grid of two-sided parameters (p, q) (Section 6.4.2,
  Figure 2).
* ``mixed_precision``: the mixed-precision workload (4096 x 8192 cells, 16 Robin
  strips, 4000 steps) run to e_mis < 1e-8 in the mixed form and in plain FP64, with
  the wall times, the iteration counts and the difference of the two results.

Every run solves the error equation of the model problem (Section 6.1: periodic in
x, zero flux in v, f = 0, u0 = 0, T = 2) on two strips split at v = 0 from a random
lambda_1^0, in the serial order SWR1-SWR4 of Section 6.3 unless ``parallel`` is set,
with the implicit-Euler/upwind scheme or (``scheme=1``) the paper's own Lie splitting
with P1 elements of Section 6.2.
The exact solution of the error equation is zero, so besides the stopping norm each
run reports the true error max |u^k(T)|: the classical algorithm without overlap
stops at once in the serial order (both strips take the same interface value, so
e_mis = 0) while its iterate stays at the initial error.

Command line::

    python -m paper_1306_4596_gb300.experiments table1 --levels 0 1 2
    python -m paper_1306_4596_gb300.experiments pscan --j 0 --p 2 8 0.25
    python -m paper_1306_4596_gb300.experiments pqscan --j 0 --p 2 14 1 --q 1 6 0.5
    python -m paper_1306_4596_gb300.experiments mixed
"""
from __future__ import annotations

import argparse
import json
import sys
import time
from typing import Dict, Iterable, List, Optional

import numpy as np

from . import inputs
from . import swr as _swr

TOL = 1e-6
MAX_ITERS = 150
# (transmission is Robin, p, q) of the three algorithms compared in Table 1
METHODS = {
    "CSWR": (False, 4.23, None),
    "OSWR(p)": (True, 4.23, None),
    "OSWR(p,q)": (True, 11.0, 2.5),
}


def _problem(j: int, overlap: int, robin: bool, p: float, q: Optional[float], parallel: bool, seed: int,
             scheme: int = 0):
    prob = inputs.model_error_equation(j, overlap=overlap, robin=robin, p=p, q=q, seed=seed)
    return prob.replace(gauss_seidel=not parallel, scheme=scheme)


def count_iterations(prob, max_iters: int = MAX_ITERS, tol: float = TOL, precision: str = "f64") -> Dict:
    """Run until e_mis < tol or max_iters; return the count, the stopping norm and the
    true error max |u(T)| of the last iterate (the exact solution is zero)."""
    t0 = time.perf_counter()
    with _swr.SWR(prob, precision) as s:
        done = s.sweep(max_iters, tol=tol, tol_kind=1)
        e_mis, e_chg, _, hist = s.error()
        true_err = float(np.abs(s.solution()).max())
    converged = bool(e_mis < tol and true_err < 100 * tol)
    return {"iters": int(done), "converged": converged, "e_mis": float(e_mis), "e_chg": float(e_chg),
            "true_error": true_err, "seconds": time.perf_counter() - t0,
            "history": [float(h[0]) for h in hist]}


def table1(levels: Iterable[int] = (0, 1, 2, 3, 4), parallel: bool = False, seed: int = 7,
           max_iters: int = MAX_ITERS, precision: str = "f64", methods: Optional[List[str]] = None,
           log=None, scheme: int = 0) -> List[Dict]:
    rows = []
    for overlap in (3, 0):
        for name in (methods or list(METHODS)):
            robin, p, q = METHODS[name]
            for j in levels:
                prob = _problem(j, overlap, robin, p, q, parallel, seed, scheme)
                # without overlap the classical algorithm cannot converge (Section 6.5):
                # a few iterations show it
                cap = min(max_iters, 10) if (overlap == 0 and not robin) else max_iters
                r = count_iterations(prob, cap, precision=precision)
                r.pop("history")
                r.update({"method": name, "overlap": overlap, "j": j, "nx": prob.nx, "nv": prob.nv,
                          "nt": prob.nt, "order": "parallel" if parallel else "serial",
                          "scheme": "split P1" if scheme == 1 else "implicit Euler + upwind"})
                rows.append(r)
                if log:
                    log(json.dumps(r))
    return rows


def format_table1(rows: List[Dict], max_iters: int = MAX_ITERS) -> str:
    levels = sorted({r["j"] for r in rows})
    out = ["| decomposition | method | " + " | ".join(f"j={j}" for j in levels) + " |",
           "|---|---|" + "---|" * len(levels)]
    for overlap in (3, 0):
        for name in METHODS:
            cells = []
            for j in levels:
                r = next((x for x in rows if x["overlap"] == overlap and x["method"] == name and x["j"] == j), None)
                if r is None:
                    cells.append("")
                elif r["converged"]:
                    cells.append(str(r["iters"]))
                elif overlap == 0 and name == "CSWR":
                    cells.append("-")
                else:
                    cells.append(f">{r['iters']}")
            label = "overlap 3 cells" if overlap else "no overlap"
            out.append(f"| {label} | {name} | " + " | ".join(cells) + " |")
    return "\n".join(out)


def p_scan(ps: Iterable[float], j: int = 0, overlap: int = 3, q: Optional[float] = None, parallel: bool = False,
           seed: int = 7, max_iters: int = MAX_ITERS, after: int = 15, precision: str = "f64",
           scheme: int = 0) -> List[Dict]:
    """Iterations to e_mis < 1e-6 and e_mis after ``after`` iterations for every p
    (q = p unless given).  One solver; the Robin factors are rebuilt in place per p."""
    ps = [float(p) for p in ps]
    prob = _problem(j, overlap, True, ps[0], q, parallel, seed, scheme)
    lam0 = prob.lam0
    out = []
    with _swr.SWR(prob, precision) as s:
        for p in ps:
            qq = p if q is None else q
            s.set_robin([p], [qq])
            s.set_traces(lam0)
            done = s.sweep(max_iters, tol=TOL, tol_kind=1)
            e_conv = s.error()[0]
            s.set_traces(lam0)
            s.sweep(after)
            hist = s.error()[3]
            out.append({"p": p, "q": qq, "iters": int(done), "converged": bool(e_conv < TOL),
                        f"e_mis_after_{after}": float(hist[-1][0])})
    return out


def pq_scan(ps: Iterable[float], qs: Iterable[float], **kw) -> List[Dict]:
    rows = []
    for q in qs:
        rows.extend(p_scan(ps, q=float(q), **kw))
    return rows


def mixed_precision(tol: float = 1e-8, max_f64: int = 400, max_mixed: int = 40, log=None) -> Dict:
    """Time to e_mis < tol on the mixed-precision workload, mixed form against plain
    FP64 (both from lambda^0 = 0, CUDA graphs, inputs on the device), plus the FP32
    per-iteration time, and the maximum differences of the two results (solution at
    T and interface data) relative to the FP64 ones."""
    import torch
    prob = inputs.mixed_precision_workload()
    out = {"workload": "Nx=4096, Nv=8192, 16 Robin strips p=4, dt=5e-5, Nt=4000, Gaussian bumps (seed 4)",
           "cell_updates_per_iteration": _swr.cell_updates_per_iteration(prob), "tol": tol}
    res = {}
    for prec, cap in (("mixed", max_mixed), ("f64", max_f64)):
        with _swr.SWR(prob, prec, inputs_on="device") as s:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.sweep(cap, tol, 1)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            e = s.error()
            cnt = s.counters()
            res[prec] = (s.solution(), s.traces())
        out[prec] = {"seconds": el, "fp64_iterations": cnt["fp64_iterations"],
                     "fp32_iterations": cnt["fp32_iterations"], "e_mis": float(e[0]), "reached": bool(e[0] < tol)}
        if log:
            log(json.dumps({prec: out[prec]}))
    with _swr.SWR(prob, "f32", inputs_on="device") as s:
        s.sweep(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.sweep(3)
        torch.cuda.synchronize()
        out["f32_seconds_per_iteration"] = (time.perf_counter() - t0) / 3
    out["f64_seconds_per_iteration"] = out["f64"]["seconds"] / max(out["f64"]["fp64_iterations"], 1)
    (um, lm), (u64, l64) = res["mixed"], res["f64"]
    out["max_rel_diff_solution"] = float(np.abs(um - u64).max() / np.abs(u64).max())
    out["max_rel_diff_traces"] = float(np.abs(lm - l64).max() / np.abs(l64).max())
    if out["mixed"]["reached"] and out["f64"]["reached"]:
        out["speedup_mixed_vs_f64"] = out["f64"]["seconds"] / out["mixed"]["seconds"]
    return out


def _range(spec: List[float]) -> np.ndarray:
    lo, hi, step = spec
    return np.round(np.arange(lo, hi + 0.5 * step, step), 10)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("table1")
    t.add_argument("--levels", type=int, nargs="+", default=[0, 1, 2, 3, 4])
    t.add_argument("--methods", nargs="+", default=None, choices=list(METHODS))
    t.add_argument("--max-iters", type=int, default=MAX_ITERS)
    mx = sub.add_parser("mixed")
    mx.add_argument("--tol", type=float, default=1e-8)
    mx.add_argument("--max-f64", type=int, default=400)
    for name in ("pscan", "pqscan"):
        sp = sub.add_parser(name)
        sp.add_argument("--j", type=int, default=0)
        sp.add_argument("--overlap", type=int, default=3)
        sp.add_argument("--p", type=float, nargs=3, default=[2.0, 8.0, 0.25], metavar=("LO", "HI", "STEP"))
        if name == "pqscan":
            sp.add_argument("--q", type=float, nargs=3, default=[1.0, 6.0, 0.5], metavar=("LO", "HI", "STEP"))
    for sp in (t, sub.choices["pscan"], sub.choices["pqscan"]):
        sp.add_argument("--parallel", action="store_true", help="parallel form instead of the serial order")
        sp.add_argument("--seed", type=int, default=7)
        sp.add_argument("--precision", default="f64", choices=["f64", "f32"])
        sp.add_argument("--scheme", type=int, default=0, choices=[0, 1],
                        help="0: implicit Euler + upwind; 1: the Lie splitting with P1 elements")
    a = ap.parse_args(argv)
    if a.cmd == "mixed":
        print(json.dumps(mixed_precision(a.tol, a.max_f64, log=lambda s: print(s, flush=True))), flush=True)
    elif a.cmd == "table1":
        rows = table1(a.levels, a.parallel, a.seed, a.max_iters, a.precision, a.methods,
                      log=lambda s: print(s, flush=True), scheme=a.scheme)
        print(format_table1(rows, a.max_iters))
    elif a.cmd == "pscan":
        for r in p_scan(_range(a.p), a.j, a.overlap, None, a.parallel, a.seed, precision=a.precision,
                        scheme=a.scheme):
            print(json.dumps(r), flush=True)
    else:
        for r in pq_scan(_range(a.p), _range(a.q), j=a.j, overlap=a.overlap, parallel=a.parallel, seed=a.seed,
                         precision=a.precision, scheme=a.scheme):
            print(json.dumps(r), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
