"""torch.autograd.Function over the ADR solve and its discrete adjoint.

``MembraneProblem`` fixes a geometry (fiber table, rates k1, k2), the flow
(solved once on the GPU; the flow does not depend on the catalysts) and the
ADR settings.  ``MembraneProblem.efficiency(w)`` returns the steady
efficiency (Eq. A-B of the paper) as a differentiable function of relaxed
per-fiber catalyst weights w_f in [0, 1] (k_AB = w_f k1, k_BC = (1 - w_f) k2
on every node of fiber f).  Its backward pass runs ``lbm_adr_adjoint``: the
transposed stream-collide iterated to its fixed point, then the chain rule
from per-node rates to per-fiber weights -- all in liblbm's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lbm


class MembraneProblem:
    def __init__(self, nx: int, ny: int, fibers, k1: float, k2: float,
                 tau_c, nspecies: int = 3, u0: float = 0.05,
                 tau_flow: float = 0.8, precision: int = lbm.LBM_F64,
                 tol: float = 1e-12, check_every: int = 500,
                 max_steps: int = 400000, flow_tol: float = 1e-10,
                 adjoint_tol: float | None = None, device="cuda"):
        self.nx, self.ny = nx, ny
        self.fibers = np.array(fibers, dtype=np.float64).reshape(-1, 6)
        self.k1, self.k2 = k1, k2
        self.nspecies = nspecies
        self.tau = list(tau_c) if hasattr(tau_c, "__len__") else \
            [tau_c] * nspecies
        self.precision = precision
        self.tol, self.check_every, self.max_steps = tol, check_every, \
            max_steps
        self.adjoint_tol = tol if adjoint_tol is None else adjoint_tol
        geom = lbm.Geometry(nx, ny, self.fibers, k1, k2).upload(device)
        flow_prec = lbm.LBM_F64 if precision == lbm.LBM_F64 else lbm.LBM_F32
        self.u, self.flow_info = lbm.lbm_flow_solve(
            geom, tau_flow, u0, max_steps, tol=flow_tol,
            check_every=check_every, precision=flow_prec)
        self.device = geom.ws.device
        self.last = None

    @property
    def nfibers(self) -> int:
        return self.fibers.shape[0]

    def solver(self, w: np.ndarray):
        fib = self.fibers.copy()
        fib[:, 5] = w
        geom = lbm.Geometry(self.nx, self.ny, fib, self.k1, self.k2).upload(
            self.device)
        prm = lbm.adr_params(self.nspecies, self.tau,
                             precision=self.precision)
        sv = lbm.ADRSolver(geom, prm, self.u).init()
        info = sv.solve(self.tol, self.check_every, self.max_steps)
        return geom, sv, info

    def efficiency(self, w: torch.Tensor) -> torch.Tensor:
        return _Efficiency.apply(w, self)


class _Efficiency(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w, prob: MembraneProblem):
        wn = w.detach().to("cpu", torch.float64).numpy()
        geom, sv, info = prob.solver(wn)
        ctx.prob = prob
        ctx.keep = (geom, sv)
        prob.last = info
        return torch.tensor(info["eps"], dtype=w.dtype, device=w.device)

    @staticmethod
    def backward(ctx, grad):
        prob = ctx.prob
        _, sv = ctx.keep
        _, _, dw, _ = sv.adjoint(prob.max_steps, tol=prob.adjoint_tol,
                                 check_every=prob.check_every,
                                 nfibers=prob.nfibers)
        ctx.keep = None
        return grad * dw.to(grad.device, grad.dtype), None
