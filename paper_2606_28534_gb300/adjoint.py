"""Gradients of the collisionless PIC run behind ``torch.autograd``.

``observables(theta, model)`` returns the tensor ``J = (J_flux, J_fe)`` of a recording forward of
``model`` (a ``pic.Adjoint``) at ``theta = (V_left, T_e)``; ``J.backward(g)`` or
``torch.autograd.grad`` then runs one reverse sweep of the library's discrete adjoint (with step
checkpointing and recomputation) for the vector-Jacobian product ``g . dJ/dtheta``.  The model
keeps the tape of its last recording forward only, so a backward must follow its own forward:
an older graph node refuses to run.
"""
from __future__ import annotations

import torch


class PicObservables(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, model):
        if theta.shape != (2,):
            raise ValueError("theta = (V_left, T_e)")
        J = model.forward(float(theta[0]), float(theta[1]))
        ctx.model = model
        ctx.recorded = model.recorded
        ctx.generation = getattr(model, "_generation", 0) + 1
        model._generation = ctx.generation
        return torch.tensor(J, dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx, gJ):
        model = ctx.model
        if getattr(model, "_generation", None) != ctx.generation or model.recorded != ctx.recorded:
            raise RuntimeError("the model ran another recording forward since this one: its tape is gone")
        g = model.gradient(float(gJ[0]), float(gJ[1]))
        return torch.tensor(g, dtype=torch.float64, device=gJ.device), None


def observables(theta: torch.Tensor, model) -> torch.Tensor:
    """(J_flux, J_fe) of a collisionless run at theta = (V_left, T_e), differentiable in theta."""
    return PicObservables.apply(theta, model)
