"""torch.autograd.Function over the adjoint of the float64 step.

rollout(solver, w0, theta, n_steps) runs n_steps steps of the step from the
primitive initial state w0 (packed layout, CUDA float64 tensor) with the
differentiable parameters theta = [G_l, sigma_y_l, Q_l for l = 0, 1] and
returns (q_final, J): the final conservative state (packed) and the running
objective J = sum_n dt_n sum_cells phi_l (rho u) dx dy of material l.
backward calls the library's checkpointed reverse sweep (dis_adjoint):
gradients with respect to w0 and theta, every time step held at the value
the forward run recorded.  All arithmetic runs in libdis.so; this module
only marshals tensors.
"""
from __future__ import annotations

import torch

from . import _lib as L


class Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w0, theta, solver, n_steps, every, material):
        if not (w0.is_cuda and w0.dtype == torch.float64):
            raise TypeError("w0 must be a CUDA float64 tensor (packed primitive state)")
        solver.set_params(theta.detach().to("cpu", torch.float64).numpy())
        solver.set_state(w0.detach().contiguous(), L.DIS_PRIMITIVE)
        J, dts = solver.adj_forward(n_steps, every=every, material=material)
        qN = torch.empty_like(w0)
        solver.get_state(L.DIS_CONSERVATIVE, out=qN)
        ctx.solver = solver
        ctx.dts = dts
        ctx.theta_meta = (theta.dtype, theta.device)
        return qN, torch.tensor(J, dtype=torch.float64, device=w0.device)

    @staticmethod
    def backward(ctx, g_qN, g_J):
        s = ctx.solver
        jbar = 0.0 if g_J is None else float(g_J)
        qbar = None if g_qN is None else g_qN.detach().contiguous().to(torch.float64)
        out = torch.empty(s.state_numel, dtype=torch.float64, device=s.device)
        g, gp = s.adjoint(qbar, jbar, kind=L.DIS_PRIMITIVE, out=out)
        dtype, dev = ctx.theta_meta
        return g, torch.as_tensor(gp, dtype=dtype, device=dev), None, None, None, None


def rollout(solver, w0, theta, n_steps, every=20, material=0):
    """(q_final, J) with gradients through the library's adjoint."""
    return Rollout.apply(w0, theta, solver, n_steps, every, material)
