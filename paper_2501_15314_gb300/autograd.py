"""``torch.autograd.Function`` wrappers around the step and its adjoint.

``ib_step`` runs one one-way step (Sec. 3.1, scalar C mode) with the marker
positions X and prescribed velocities U^Gamma as differentiable inputs; its
backward is one call of ``ibm_adjoint_step`` (a transposed Schur solve, plus a
predictor solve when F^n is nonzero).  ``body_loads`` gives per body the IB
force h^3 sum F_k (Eq. (IBM_force)) and torque h^3 sum (X_k - c) x F_k, with
backward ``ibm_body_forces_adjoint``.  The body feels minus these (the
direct-forcing term acts on the fluid), so the drag-plus-torque loss of a body
is ``-(loads[b, 2] + loads[b, 5])``.

Only the force F^{n+1} carries gradients; u^{n+1} and p^{n+1} are returned
as non-differentiable, and the state (u^n, u^{n-1}, p^n, F^n, f) is a
constant of the step.
"""
from __future__ import annotations

import numpy as np
import torch

__all__ = ["ib_step", "body_loads"]


class _StepForce(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, U_gamma, solver, state, opts):
        Xd = X.detach().contiguous()
        solver.set_markers(Xd)
        out, st = solver.step(state["u_n"], state["u_nm1"], state["p_n"], state["F_n"],
                              U_gamma.detach().contiguous(), state.get("f_body"), **opts)
        ctx.solver, ctx.opts, ctx.F_n = solver, opts, state["F_n"]
        ctx.save_for_backward(Xd, out["u"], out["F"])
        ctx.mark_non_differentiable(out["u"], out["p"])
        solver.last_step_stats = st
        return out["F"], out["u"], out["p"]

    @staticmethod
    def backward(ctx, F_bar, u_bar, p_bar):
        X, u_np1, F_np1 = ctx.saved_tensors
        s = ctx.solver
        s.set_markers(X)   # another forward may have moved the markers since
        U_bar, X_bar, st = s.adjoint_step(u_np1, ctx.F_n, F_np1, F_bar.contiguous(), **ctx.opts)
        s.last_adjoint_stats = st
        return X_bar.view_as(X), U_bar, None, None, None


class _BodyLoads(torch.autograd.Function):
    @staticmethod
    def forward(ctx, F, X, centers, solver, body_id):
        c_np = centers.detach().cpu().numpy().astype(np.float64).reshape(-1, 3)
        out = solver.body_forces(F.detach().contiguous(), X.detach().contiguous().view(-1),
                                 body_id, c_np)
        ctx.solver, ctx.body_id, ctx.c_np, ctx.out = solver, body_id, c_np, out
        ctx.c_device = centers.device
        ctx.save_for_backward(F.detach(), X.detach())
        return torch.from_numpy(out)

    @staticmethod
    def backward(ctx, g):
        F, X = ctx.saved_tensors
        F_bar, X_bar, c_bar = ctx.solver.body_forces_adjoint(
            F.contiguous(), X.contiguous().view(-1), ctx.body_id, ctx.c_np,
            g.detach().cpu().numpy(), ctx.out)
        return (F_bar.view_as(F), X_bar.view_as(X),
                torch.from_numpy(c_bar).to(ctx.c_device), None, None)


def ib_step(solver, X, U_gamma, state, **opts):
    """One step with differentiable X ((3, N) CUDA float64) and U_gamma
    ((3N,) CUDA float64).  state: dict of u_n, u_nm1, p_n, F_n and optional
    f_body (CUDA float64).  Returns (F^{n+1}, u^{n+1}, p^{n+1})."""
    return _StepForce.apply(X, U_gamma, solver, state, opts)


def body_loads(solver, F, X, body_id, centers):
    """Per-body [IB force | IB torque] as a (n_bodies, 6) CPU float64 tensor,
    differentiable in F, X and centers ((n_bodies, 3), any device)."""
    return _BodyLoads.apply(F, X, centers, solver, body_id)
