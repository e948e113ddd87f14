"""Differentiation of K SWR iterations with respect to the Robin parameters.

``InterfaceMismatch`` is a ``torch.autograd.Function`` whose forward runs K
iterations on the GPU and returns J = dt hx sum (u_j - u_{j+1})^2 on the interface
nodes of the K-th iterate, and whose backward returns the gradient computed by the
library's hand-written discrete adjoint (``kfp_swr_gradient``): the transposed
implicit-Euler systems solved backward in time and the transposed exchange backward
over the iterates.  ``optimize_robin`` minimises J over the per-interface parameters
(one-sided: q = p, the optimized Schwarz method OSWR(p) of Section 6.4) with Adam on
log p, the numerical counterpart of the paper's sampling search for p*.
"""
from __future__ import annotations

from typing import List, Optional

import numpy as np


def _torch():
    import torch
    return torch


class InterfaceMismatch:
    """Namespace for the autograd function (built lazily so that importing this
    module does not require torch)."""

    _fn = None

    @classmethod
    def fn(cls):
        if cls._fn is None:
            torch = _torch()

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, p, q, solver, K, lam0):
                    solver.set_robin(p.detach().cpu().numpy(), q.detach().cpu().numpy())
                    J, gp, gq = solver.gradient(K, lam0)
                    ctx.save_for_backward(torch.as_tensor(gp, dtype=p.dtype), torch.as_tensor(gq, dtype=q.dtype))
                    return torch.tensor(J, dtype=p.dtype)

                @staticmethod
                def backward(ctx, gJ):
                    gp, gq = ctx.saved_tensors
                    return gJ * gp, gJ * gq, None, None, None

            cls._fn = _F
        return cls._fn


def interface_mismatch(p, q, solver, K: int, lam0: Optional[np.ndarray] = None):
    """J(p, q) after K iterations, differentiable in p and q (torch tensors, FP64, CPU)."""
    return InterfaceMismatch.fn().apply(p, q, solver, K, lam0)


def optimize_robin(solver, K: int, steps: int = 20, lr: float = 0.1, p0: Optional[np.ndarray] = None) -> dict:
    """Adam on log p_j (q = p) minimising J after K iterations from zero interface data."""
    torch = _torch()
    p_init = np.array(solver.prob.p if p0 is None else p0, dtype=np.float64)
    logp = torch.tensor(np.log(p_init), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([logp], lr=lr)
    history: List[dict] = []
    for it in range(steps):
        opt.zero_grad()
        p = torch.exp(logp)
        J = interface_mismatch(p, p, solver, K)
        J.backward()
        history.append({"step": it, "J": float(J.item()), "p": p.detach().numpy().tolist()})
        opt.step()
    p = torch.exp(logp).detach()
    J = interface_mismatch(p, p, solver, K)
    history.append({"step": steps, "J": float(J.item()), "p": p.numpy().tolist()})
    return {"p": p.numpy(), "J": float(J.item()), "history": history}
