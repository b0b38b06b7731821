"""Gradients of moment-based losses with respect to the SMRT relaxation times, through
torch.autograd, on libsmrt's adjoint kernels (lb_step_adjoint, lb_moments_adjoint).

``relaxation_run(ctx, tau, h0, nsteps, ...)`` returns the moments (lb_moments rows) of the
state after nsteps collide-and-stream steps started from h0 with continuous relaxation times
tau (one per irreducible part (n, m), lb_set_relaxation's order). Its backward pass runs the
discrete adjoint with step checkpointing: the forward pass keeps every ``checkpoint_every``-th
state on the device; the backward pass recomputes each segment's states from its checkpoint and
walks them in reverse. The gradient with respect to tau is accumulated in double.
"""
from __future__ import annotations

import torch

from . import api
from ._ffi import LB_MOM_Q, LB_MOM_RHO, LB_MOM_THETA

SHOCK_LOSS_MASK = LB_MOM_RHO | LB_MOM_THETA | LB_MOM_Q


class _RelaxationRun(torch.autograd.Function):
    @staticmethod
    def forward(fctx, tau, ctx, h0, nsteps, checkpoint_every, mask):
        args = dict(ctx.relax_args)
        api.lb_set_relaxation(ctx, tau.detach().cpu().double().numpy(), **args)
        fa, fb = ctx.new_state(), ctx.new_state()
        fa.copy_(h0)
        ckpts = {0: h0.clone()}
        cur, other = fa, fb
        for t in range(nsteps):
            cur = api.lb_step(ctx, cur, other, 1)
            other = fa if cur is fb else fb
            if (t + 1) % checkpoint_every == 0 and t + 1 < nsteps:
                ckpts[t + 1] = cur.clone()
        final = cur.clone()
        out = api.lb_moments(ctx, final, mask)
        fctx.lbctx = ctx
        fctx.ckpts = ckpts
        fctx.final = final
        fctx.nsteps = nsteps
        fctx.every = checkpoint_every
        fctx.mask = mask
        fctx.tau = tau.detach().cpu().double().numpy()
        fctx.tau_dtype = tau.dtype
        return out

    @staticmethod
    def backward(fctx, gout):
        ctx = fctx.lbctx
        api.lb_set_relaxation(ctx, fctx.tau, **ctx.relax_args)
        lam = torch.empty(ctx.state_elems, dtype=torch.float64, device=ctx.device)
        lam2 = torch.empty_like(lam)
        api.lb_moments_adjoint(ctx, fctx.final, gout.contiguous().double(), fctx.mask, lam)
        dtau = torch.zeros(len(fctx.tau), dtype=torch.float64, device=ctx.device)
        starts = sorted(fctx.ckpts)
        for s0 in reversed(starts):
            s1 = min(s0 + fctx.every, fctx.nsteps)
            states = [fctx.ckpts[s0]]
            fa, fb = ctx.new_state(), ctx.new_state()
            cur, other = states[0], fa
            for _ in range(s0, s1 - 1):
                nxt = api.lb_step(ctx, cur, other, 1)
                states.append(nxt.clone())
                cur, other = nxt, (fb if nxt is fa else fa)
            for t in range(s1 - 1, s0 - 1, -1):
                api.lb_step_adjoint(ctx, states[t - s0], lam, lam2, dtau)
                lam, lam2 = lam2, lam
        return dtau.cpu().to(fctx.tau_dtype), None, None, None, None, None


def relaxation_run(ctx, tau, h0, nsteps: int, checkpoint_every: int = 250, mask: int = SHOCK_LOSS_MASK):
    """Moments after nsteps steps from h0, differentiable with respect to tau (CPU tensor)."""
    return _RelaxationRun.apply(tau, ctx, h0, int(nsteps), int(checkpoint_every), int(mask))
