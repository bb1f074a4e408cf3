"""Differentiable residual and two-stage fourth-order time stepping.

GKSResidual wraps gks_residual (forward) and gks_residual_vjp (backward), and S2O4Stage wraps
gks_s2o4_stage and its transpose gks_s2o4_stage_vjp, each in a torch.autograd.Function; every
operation of the rollout runs in the library's kernels, and this module only wires the calls.
s2o4_rollout advances a state through n S2O4 steps of Section 3.3
  Q* = Q + dt/2 L(Q) + dt^2/8 Lt(Q),  Q' = Q + dt L(Q) + dt^2/6 (Lt(Q) + 2 Lt(Q*))
with checkpoints every k steps (torch.utils.checkpoint): the backward pass recomputes one segment
at a time, so memory holds the checkpoints plus one segment's stage states.
"""
from __future__ import annotations

import torch
from torch.utils.checkpoint import checkpoint

from . import gks_residual, gks_residual_vjp, gks_s2o4_stage, gks_s2o4_stage_vjp


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


class GKSResidual(torch.autograd.Function):
    """(L, Lt) = residual(Q) for a fixed dt; Q is float64 [5, n_cells] on the solver's device."""

    @staticmethod
    def forward(ctx, Q, solver, dt):
        Q = Q.contiguous()
        L = torch.empty_like(Q)
        Lt = torch.empty_like(Q)
        gks_residual(solver.h, Q, dt, L, Lt)
        ctx.save_for_backward(Q)
        ctx.solver = solver
        ctx.dt = dt
        return L, Lt

    @staticmethod
    def backward(ctx, gL, gLt):
        (Q,) = ctx.saved_tensors
        gL = torch.zeros_like(Q) if gL is None else gL.contiguous()
        gLt = torch.zeros_like(Q) if gLt is None else gLt.contiguous()
        gQ = torch.empty_like(Q)
        gks_residual_vjp(ctx.solver.h, Q, ctx.dt, gL, gLt, gQ)
        return gQ, None, None


class S2O4Stage(torch.autograd.Function):
    """Stage 1: Q + dt/2 L + dt^2/8 Lt; stage 2: Q + dt L + dt^2/6 (Lt + 2 Lts)."""

    @staticmethod
    def forward(ctx, Q, L, Lt, Lts, stage, dt):
        Q, L, Lt = Q.contiguous(), L.contiguous(), Lt.contiguous()
        Lts = None if Lts is None else Lts.contiguous()
        out = torch.empty_like(Q)
        gks_s2o4_stage(stage, dt, Q, L, Lt, Lts, out, _stream())
        ctx.stage, ctx.dt = stage, dt
        return out

    @staticmethod
    def backward(ctx, g):
        g = g.contiguous()
        gQ, gL, gLt = torch.empty_like(g), torch.empty_like(g), torch.empty_like(g)
        gLts = torch.empty_like(g) if ctx.stage == 2 else None
        gks_s2o4_stage_vjp(ctx.stage, ctx.dt, g, gQ, gL, gLt, gLts, _stream())
        return gQ, gL, gLt, gLts, None, None


def s2o4_step(Q, solver, dt):
    L, Lt = GKSResidual.apply(Q, solver, dt)
    Qs = S2O4Stage.apply(Q, L, Lt, None, 1, dt)
    _, Lts = GKSResidual.apply(Qs, solver, dt)
    return S2O4Stage.apply(Q, L, Lt, Lts, 2, dt)


def _segment(Q, solver, dt, n):
    for _ in range(n):
        Q = s2o4_step(Q, solver, dt)
    return Q


def s2o4_rollout(Q0, solver, dt, nsteps, checkpoint_every=20):
    """Differentiable n-step S2O4 rollout with a checkpoint every `checkpoint_every` steps."""
    Q = Q0
    done = 0
    while done < nsteps:
        n = min(checkpoint_every, nsteps - done)
        if torch.is_grad_enabled() and Q.requires_grad:
            Q = checkpoint(_segment, Q, solver, dt, n, use_reentrant=False)
        else:
            Q = _segment(Q, solver, dt, n)
        done += n
    return Q
