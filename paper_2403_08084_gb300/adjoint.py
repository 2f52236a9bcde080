"""Differentiation through the RK time loop (torch.autograd), by the library's discrete adjoint.

``trajectory(solver, theta, u0, steps, ...)`` returns u_N as a function of the
per-cell log-diffusivity theta = log(kappa).  Its backward pass is the exact
discrete adjoint of the forward loop: every ``irk_step`` has a matching
``irk_step_adjoint`` (transposed stage system, transposed preconditioner).  The
forward pass keeps the state only every ``checkpoint`` steps; the backward pass
re-runs each segment forward to regenerate the states and stages it needs and
then walks that segment in reverse.  ``mass_norm2`` gives 1/2 e^T M e with its
gradient M e.  All arithmetic runs in libirk.so; this module only sequences the
calls.
"""
from __future__ import annotations

import torch


def _coef(f_coef, n):
    return None if f_coef is None else list(f_coef(n))


class _Trajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, u0, solver, steps, f_space, f_coef, checkpoint, allow_noconv):
        solver.set_kappa(torch.exp(theta.detach()).cpu().numpy())
        u = u0.detach().clone().contiguous()
        ckpt = {0: u.clone()}
        for n in range(steps):
            solver.step(u, u, f_space=f_space, f_coef=_coef(f_coef, n), allow_noconv=allow_noconv)
            if (n + 1) % checkpoint == 0 and n + 1 < steps:
                ckpt[n + 1] = u.clone()
        ctx.solver, ctx.steps, ctx.f_space, ctx.f_coef, ctx.ckpt = solver, steps, f_space, f_coef, ckpt
        ctx.allow_noconv = allow_noconv
        ctx.save_for_backward(theta)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (theta,) = ctx.saved_tensors
        sv = ctx.solver
        sv.set_kappa(torch.exp(theta.detach()).cpu().numpy())
        lam = grad_u.detach().clone().contiguous()
        grad = torch.zeros(sv.n_cells, dtype=torch.float64, device=lam.device)
        starts = sorted(ctx.ckpt)
        ends = starts[1:] + [ctx.steps]
        sv.adjoint_its = []  # Krylov iterations of every adjoint solve, in the order they ran
        for a, b in reversed(list(zip(starts, ends))):
            # regenerate the segment's states and stages
            us, ks = [ctx.ckpt[a].clone()], []
            for n in range(a, b):
                u1 = torch.empty_like(us[-1])
                k = torch.empty(sv.n_nodes * sv.s, dtype=torch.float64, device=lam.device)
                sv.step(us[-1], u1, f_space=ctx.f_space, f_coef=_coef(ctx.f_coef, n), stages_out=k,
                        allow_noconv=ctx.allow_noconv)
                us.append(u1)
                ks.append(k)
            for n in range(b - 1, a - 1, -1):
                st = sv.step_adjoint(us[n - a], ks[n - a], lam, lam, grad, allow_noconv=ctx.allow_noconv)
                sv.adjoint_its.append(st["fgmres_its"])
        return grad.to(theta.dtype), lam, None, None, None, None, None, None


def trajectory(solver, theta, u0, steps, f_space=None, f_coef=None, checkpoint=10, allow_noconv=False):
    """u_N after ``steps`` RK steps from u0 with kappa = exp(theta) (differentiable in theta and u0).

    f_space: nodal load vector (device tensor) or None; f_coef(n) -> s per-stage factors for step n.
    allow_noconv: accept FGMRES solves that stop at maxit (a fixed iteration count makes u_N a
    smooth function of theta, which finite-difference checks need).
    """
    return _Trajectory.apply(theta, u0, solver, int(steps), f_space, f_coef, int(checkpoint), bool(allow_noconv))


class _MassNorm2(torch.autograd.Function):
    @staticmethod
    def forward(ctx, e, solver):
        Me = torch.empty_like(e)
        solver.apply_mass(e.detach().contiguous(), Me)
        ctx.save_for_backward(Me)
        return 0.5 * torch.dot(e.detach(), Me)

    @staticmethod
    def backward(ctx, g):
        (Me,) = ctx.saved_tensors
        return g * Me, None


def mass_norm2(solver, e):
    """1/2 e^T M e for a nodal vector e (differentiable)."""
    return _MassNorm2.apply(e, solver)
