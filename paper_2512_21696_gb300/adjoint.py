"""Porosity gradient behind ``torch.autograd``: the loss of a run as a
differentiable function of the per-cell porosity, with the library's
hand-written adjoint (``lbm_adjoint_run``) as its backward.

    loss = porosity_loss(phi, ctx, cell, rhoA, rhoB, nsteps=..., ckpt=100,
                         q_target=..., s_target=..., pore_type=None)
    loss.backward()          # phi.grad = dL/dphi (zero outside gray cells)

Each call sets the geometry from ``phi`` (gray cells), initialises the fields
from rhoA/rhoB and runs nsteps forward steps with checkpoints every ckpt
steps; the gradient is computed in the same call and handed to autograd.
"""
from __future__ import annotations

import numpy as np

from . import lbm


def _torch():
    import torch
    return torch



def _make_function():
    torch = _torch()

    class PorosityLoss(torch.autograd.Function):
        @staticmethod
        def forward(actx, phi, ctx, cell, rhoA, rhoB, pore_type, nsteps, ckpt, q_target, s_target):
            ph = phi.detach().to(torch.float32).contiguous()
            lbm.lbm_set_geometry(ctx, cell, ph, pore_type)
            lbm.lbm_init_fields(ctx, rhoA, rhoB)
            if ph.is_cuda:
                grad = torch.empty_like(ph)
                loss, q, S, _ = lbm.lbm_adjoint_run(ctx, q_target, s_target, nsteps, ckpt, grad)
            else:
                loss, q, S, g = lbm.lbm_adjoint_run(ctx, q_target, s_target, nsteps, ckpt)
                grad = torch.from_numpy(g)
            actx.save_for_backward(grad)
            actx.q, actx.S = q, S
            return torch.tensor(loss, dtype=torch.float64, device=phi.device)

        @staticmethod
        def backward(actx, g):
            (grad,) = actx.saved_tensors
            return (g.to(grad.dtype) * grad).to(g.device), None, None, None, None, None, None, None, None, None

    return PorosityLoss


_FN = None


def porosity_loss(phi, ctx, cell, rhoA, rhoB, nsteps, ckpt, q_target, s_target, pore_type=None):
    """L(phi) as a torch scalar whose backward is the hand-written adjoint."""
    global _FN
    if _FN is None:
        _FN = _make_function()
    return _FN.apply(phi, ctx, cell, rhoA, rhoB, pore_type, int(nsteps), int(ckpt), float(q_target),
                     float(s_target))
