"""Differentiable multi-step evolution: torch.autograd.Function over mhd_step / mhd_step_adjoint.

The forward pass runs the steps with a given (frozen) dt sequence and keeps the state every
`every` steps; the backward pass recomputes each segment from its checkpoint and runs the
library's hand-written adjoint step by step in reverse. Gradients flow to the initial conserved
state, the initial face field and eta; anything upstream of those (for example an initial
velocity field turned into momentum and energy with torch operations) is handled by autograd.
Steps in which flux correction replaced fluxes are differentiated with the flagged cells held
fixed, like every other branch of the step.
"""
from __future__ import annotations

import torch

from . import mhd


class MHDEvolve(torch.autograd.Function):
    @staticmethod
    def forward(fctx, cons0, b0, eta, ctx: mhd.Context, dts, scheme: int, every: int = 5):
        every = max(1, int(every))
        etaf = float(eta)
        st = mhd.State(cons0.detach().contiguous().clone(), b0.detach().contiguous().clone())
        ckpts = [(st.cons.clone(), st.b.clone())]
        for n, dt in enumerate(dts):
            ctx.step(st, float(dt), scheme, etaf)
            if (n + 1) % every == 0 and n + 1 < len(dts):
                ckpts.append((st.cons.clone(), st.b.clone()))
        fctx.mctx, fctx.dts, fctx.scheme, fctx.every, fctx.eta = ctx, list(dts), scheme, every, etaf
        fctx.ckpts = ckpts
        return st.cons, st.b

    @staticmethod
    def backward(fctx, gcons, gb):
        ctx, dts, scheme, every, eta = fctx.mctx, fctx.dts, fctx.scheme, fctx.every, fctx.eta
        c0, b0 = fctx.ckpts[0]
        lam = mhd.State(torch.zeros_like(c0) if gcons is None else gcons.contiguous().clone(),
                        torch.zeros_like(b0) if gb is None else gb.contiguous().clone())
        deta = 0.0
        for k in reversed(range(len(fctx.ckpts))):
            n0, n1 = k * every, min((k + 1) * every, len(dts))
            st = mhd.State(fctx.ckpts[k][0].clone(), fctx.ckpts[k][1].clone())
            states = [(st.cons.clone(), st.b.clone())]
            for n in range(n0, n1 - 1):  # recompute the segment's states from its checkpoint
                ctx.step(st, float(dts[n]), scheme, eta)
                states.append((st.cons.clone(), st.b.clone()))
            for n in reversed(range(n0, n1)):
                s = mhd.State(*states[n - n0])
                deta += ctx.step_adjoint(s, lam, float(dts[n]), scheme, eta)
        return lam.cons, lam.b, torch.tensor(deta, dtype=torch.float64), None, None, None, None


def evolve(cons0, b0, eta, ctx: mhd.Context, dts, scheme: int, every: int = 5):
    """Final (cons, b) after len(dts) steps; differentiable w.r.t. cons0, b0 and eta (a tensor)."""
    return MHDEvolve.apply(cons0, b0, eta, ctx, dts, scheme, every)
