"""torch.autograd.Function over the ensemble-mean energy and virial.

EnsembleUW.apply(theta, system, r_all, q_all) -> tensor([<U>, <W>]) where theta
holds the force-field parameters (per LJ type eps then sigma, then every
charge, dipole and quadrupole moment; see md_set_params) and the mean runs
over the fixed configurations r_all (n_cfg x n x 3), q_all (n_cfg x n x 4).

forward runs md_param_grad once: its kernel recomputes every pair term of
every configuration and returns the means together with their parameter
derivatives, which backward contracts with the incoming gradient.  All
arithmetic runs in the CUDA library; this module only marshals.
"""
from __future__ import annotations

import numpy as np
import torch

from . import md


class EnsembleUW(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, system: "md.System", r_all, q_all):
        system.set_params(theta.detach().to("cpu", torch.float64).numpy())
        dU, dW, U, W = system.param_grad(r_all, q_all)
        ctx.dU, ctx.dW = dU, dW
        return torch.tensor([U, W], dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx, g):
        gc = g.detach().to("cpu", torch.float64).numpy()
        grad = gc[0] * ctx.dU + gc[1] * ctx.dW
        return torch.from_numpy(np.ascontiguousarray(grad)).to(g.device), None, None, None


def ensemble_uw(theta, system, r_all, q_all):
    return EnsembleUW.apply(theta, system, r_all, q_all)
