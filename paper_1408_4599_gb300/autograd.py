"""torch.autograd.Function over the ensemble-mean energy and virial.

EnsembleUW.apply(theta, system, r_all, q_all) -> tensor([<U>, <W>]) where theta
holds the force-field parameters (per LJ type eps then sigma, then every
charge, dipole and quadrupole moment; see md_set_params) and the mean runs
over the fixed configurations r_all (n_cfg x n x 3), q_all (n_cfg x n x 4).

forward evaluates the configurations with the force kernel (through
md_compute_forces / md_energy_virial); backward calls md_param_grad, whose
kernel recomputes every pair term -- nothing is stored between the two.
All arithmetic runs in the CUDA library; this module only marshals.
"""
from __future__ import annotations

import numpy as np
import torch

from . import md


class EnsembleUW(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, system: "md.System", r_all, q_all):
        th = theta.detach().to("cpu", torch.float64).numpy()
        system.set_params(th)
        U = W = 0.0
        n_cfg = r_all.shape[0]
        for c in range(n_cfg):
            system.set(r_all[c], q_all[c])
            system.compute_forces()
            o = system.observables()
            U += o["U_pot"] + o["U_lrc"]
            W += o["W"] + o["W_lrc"]
        ctx.system = system
        ctx.r_all, ctx.q_all = r_all, q_all
        ctx.theta = th
        return torch.tensor([U / n_cfg, W / n_cfg], dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx, g):
        ctx.system.set_params(ctx.theta)
        dU, dW, _, _ = ctx.system.param_grad(ctx.r_all, ctx.q_all)
        gc = g.detach().to("cpu", torch.float64).numpy()
        grad = gc[0] * dU + gc[1] * dW
        return torch.from_numpy(np.ascontiguousarray(grad)).to(g.device), None, None, None


def ensemble_uw(theta, system, r_all, q_all):
    return EnsembleUW.apply(theta, system, r_all, q_all)
