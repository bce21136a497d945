"""Differentiable supernova pass: torch.autograd.Function around the C ABI.

feedback_pass(state, particles, params, box) runs one supernova pass
(pmp_gather, pmp_deposit, pmp_fold_ghosts, pmp_apply_limited) on a copy of
``state`` and returns the updated state.  Its backward calls pmp_backward,
the hand-written adjoint: a weighted gather over the same kernel cells
(recomputed from the pass's plan), with the limited apply differentiated at
fixed eta and cells where the limiter acted passing no gradient.  Gradients
flow to the particle masses, energies, momenta and positions; the state is
treated as a constant.
"""
from __future__ import annotations

import torch

from . import pmp

_FIELDS = ("m", "e", "px", "py", "pz", "x", "y", "z")


class _FeedbackPass(torch.autograd.Function):
    @staticmethod
    def forward(ctx, state, params, box, periodic, dx, mode, m, e, px, py, pz, x, y, z):
        parts = {"m": m.detach().contiguous(), "e": e.detach().contiguous(), "px": px.detach().contiguous(),
                 "py": py.detach().contiguous(), "pz": pz.detach().contiguous(), "x": x.detach().contiguous(),
                 "y": y.detach().contiguous(), "z": z.detach().contiguous()}
        u_old = state.detach().contiguous()
        u_new = u_old.clone()
        ps = pmp.Pass(params, box, u_new, parts, mode=mode, dx=dx, periodic=periodic)
        ps.run()
        ctx.ps, ctx.parts, ctx.box, ctx.periodic, ctx.dx = ps, parts, box, periodic, dx
        ctx.save_for_backward(u_old)
        return u_new

    @staticmethod
    def backward(ctx, g_new):
        (u_old,) = ctx.saved_tensors
        ps = ctx.ps
        n = ctx.parts["x"].numel()
        gU = g_new.contiguous()
        g_out = torch.zeros((8, n), dtype=torch.float64, device=u_old.device)
        state_in = pmp.Mesh(u_old, ctx.box.n, ctx.box.g, ctx.periodic, ctx.dx)
        pmp.pmp_backward(ps.ctx, state_in, ps.buffer, ctx.parts, ps.gathered_view(), gU, g_out, ps.workspace)
        grads = [g_out[i] for i in range(8)]
        return (None, None, None, None, None, None, *grads)


def feedback_pass(state, particles, params, box, periodic=(1, 1, 1), dx=1.0, mode="atomic"):
    """One differentiable supernova pass; returns the updated state tensor."""
    args = [particles[k] for k in _FIELDS]
    return _FeedbackPass.apply(state, params, box, tuple(periodic), float(dx), mode, *args)
