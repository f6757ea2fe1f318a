"""Differentiable leapfrog rollout over the library's adjoint kernels.

``rollout(nb, x0, v0, m, G, eps, dt, nsteps, every)`` runs ``nsteps``
kick-drift-kick steps (the reading of the paper's "Move_bodies", Sec. IV-B)
and returns the final positions and velocities as tensors that torch
autograd can differentiate with respect to x0, v0 and m.

Forward: one ``nb_rollout`` call that records the state every ``every``
steps (segment checkpoints).  Backward, segment by segment from the last:
restore the checkpoint, recompute the segment's positions with
``nb_rollout(record_every=1)``, then run ``nb_step_backward`` (the reverse
sweep with the force VJP kernel).  Memory: (nsteps/every + 1) checkpoints of
(x, v) plus one segment of positions; compute: one extra forward pass.

This module only allocates tensors and orders library calls; all arithmetic
runs in the CUDA kernels.
"""
from __future__ import annotations

import torch

from .nbody import NBody


class NBodyRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, v0, m, nb: NBody, G: float, eps: float, dt: float, nsteps: int,
                every: int):
        every = max(1, int(every))
        nsteps = int(nsteps)
        n = m.shape[0]
        x = torch.empty_like(x0).copy_(x0.detach())
        v = torch.empty_like(v0).copy_(v0.detach())
        md = m.detach().contiguous()
        acc = torch.empty_like(x)
        nrec = nsteps // every + 1
        ckx = torch.empty((nrec, n, 3), dtype=x.dtype, device=x.device)
        ckv = torch.empty_like(ckx)
        if nsteps > 0:
            nb.rollout(x, v, md, G, eps, dt, nsteps, acc, every, ckx, ckv)
        ctx.nb, ctx.G, ctx.eps, ctx.dt, ctx.nsteps, ctx.every = nb, G, eps, dt, nsteps, every
        ctx.save_for_backward(ckx, ckv, md)
        return x, v

    @staticmethod
    def backward(ctx, gx, gv):
        ckx, ckv, m = ctx.saved_tensors
        nb, G, eps, dt, nsteps, every = ctx.nb, ctx.G, ctx.eps, ctx.dt, ctx.nsteps, ctx.every
        n = m.shape[0]
        lam_x = torch.zeros((n, 3), dtype=m.dtype, device=m.device)
        lam_v = torch.zeros_like(lam_x)
        if gx is not None:
            lam_x.copy_(gx)
        if gv is not None:
            lam_v.copy_(gv)
        lam_m = torch.zeros_like(m)
        if nsteps == 0:
            return lam_x, lam_v, lam_m, None, None, None, None, None, None
        nseg = (nsteps + every - 1) // every
        traj = torch.empty((every + 1, n, 3), dtype=m.dtype, device=m.device)
        x = torch.empty((n, 3), dtype=m.dtype, device=m.device)
        v = torch.empty_like(x)
        acc = torch.empty_like(x)
        for s in range(nseg - 1, -1, -1):
            start = s * every
            length = min(every, nsteps - start)
            x.copy_(ckx[s])
            v.copy_(ckv[s])
            seg = traj[: length + 1]
            nb.rollout(x, v, m, G, eps, dt, length, acc, 1, seg)
            nb.step_backward(seg, m, G, eps, dt, length, lam_x, lam_v, lam_m,
                             at_start=(s == 0), at_end=(s == nseg - 1))
        return lam_x, lam_v, lam_m, None, None, None, None, None, None


def rollout(nb: NBody, x0, v0, m, G: float, eps: float, dt: float, nsteps: int, every: int = 20):
    """Final (x, v) after nsteps leapfrog steps, differentiable in (x0, v0, m)."""
    return NBodyRollout.apply(x0, v0, m, nb, G, eps, dt, nsteps, every)
