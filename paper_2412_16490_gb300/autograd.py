"""torch.autograd binding of the grasp energy (Sec. IV-A).

Forward: the fused evaluation kernel solves the s lower-level QPs at the
poses and returns E [B].  Backward: the hand-written adjoint kernel
(`bodex_energy_adjoint`) recomputes kinematics and the SDF query from the
saved poses and applies the envelope theorem -- the QPs' feasible set does
not depend on x, so dQ_j/dG = -2 r_j y_j^T at the saved forces y_j -- down
through the contact frames and the kinematic chain.  Only x and y are saved.
"""
from __future__ import annotations

import torch

from . import bodex_energy_adjoint, bodex_energy_grad


class GraspEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, hand, obj, T, params):
        xd = x.detach().contiguous()
        out = bodex_energy_grad(hand, obj, xd, T, params)
        ctx.save_for_backward(xd, out["y"])
        ctx.hand, ctx.obj, ctx.T, ctx.params = hand, obj, T, params
        return out["E"]

    @staticmethod
    def backward(ctx, gE):
        x, y = ctx.saved_tensors
        adj = bodex_energy_adjoint(ctx.hand, ctx.obj, x, ctx.T, ctx.params, y)
        return gE.unsqueeze(1) * adj["dEdx"], None, None, None, None


def grasp_energy(x, hand, obj, T, params):
    """E [B] at poses x [B, 6+n] (CUDA float32), differentiable in x."""
    return GraspEnergy.apply(x, hand, obj, T, params)
