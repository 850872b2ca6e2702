"""Receiver misfit as a differentiable function of the per-cell wave speed.

MisfitFunction wraps the library's discrete adjoint (imex_adjoint): the
forward evaluates J(c) = 1/2 sum_n sum_cols sum_r (u_n[rec_r] - d)^2 for a
workload with wave speeds c (one context built for c, stepped from the zero
initial state), and the backward returns dJ/dc from the adjoint sweep of the
same call.  One column per source (the sources are independent right-hand
sides).
"""
import dataclasses

import numpy as np
import torch

from . import imex


def _context(w, c):
    w2 = dataclasses.replace(w, cell_c=np.asarray(c, dtype=np.float64))
    ncols = len(w.src_pos)
    return imex.Imex.from_workload(w2, ncols=ncols)


def misfit_and_gradient(w, c, rec_nodes, data, nsteps, checkpoint_every=100, dt=None):
    """(J, dJ/dc) for wave speeds c (one value per cell).  dt fixes the time
    step (the default derives it from the uncut cells of this c)."""
    w2 = w if dt is None else dataclasses.replace(w, dt=float(dt))
    with _context(w2, c) as g:
        return g.adjoint(nsteps, rec_nodes, data, checkpoint_every)


def traces(w, c, rec_nodes, nsteps, dt=None):
    """Receiver traces (nsteps x ncols x nrec) of the forward run for speeds c."""
    w2 = w if dt is None else dataclasses.replace(w, dt=float(dt))
    rec = np.ascontiguousarray(np.asarray(rec_nodes, dtype=np.int64))
    with _context(w2, c) as g:
        out = np.zeros((nsteps, g.ncols * len(rec)))
        g.step_io(nsteps, None, rec, out)
    return out.reshape(nsteps, g.ncols, len(rec))


class MisfitFunction(torch.autograd.Function):
    """J(c) with dJ/dc from the discrete adjoint; c is a float64 CPU tensor."""

    @staticmethod
    def forward(ctx, c, w, rec_nodes, data, nsteps, checkpoint_every, dt):
        J, grad = misfit_and_gradient(w, c.detach().cpu().numpy(), rec_nodes, data, nsteps,
                                      checkpoint_every, dt)
        ctx.save_for_backward(torch.from_numpy(grad))
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        (grad,) = ctx.saved_tensors
        return gJ * grad, None, None, None, None, None, None


def misfit(c, w, rec_nodes, data, nsteps, checkpoint_every=100, dt=None):
    return MisfitFunction.apply(c, w, rec_nodes, data, nsteps, checkpoint_every, dt)
