"""torch.autograd.Function over the adjoint of the fused step (lbkm_grad).

``DetonationObjective.apply(rho0, S, Q, omega1, setup)`` runs the 1-D FP64 model
from the equilibrium start (rho0, u0, T0, lambda0) for ``setup["steps"]`` steps
and returns J = w_mismatch/2 sum (rho_N - rho*)^2 dx + w_tne sum_n sum_x d_n^2 dx dt.
Its backward hands back the gradients the CUDA adjoint computed with the forward
(gradients of J with respect to rho0, the 16 rates S, Q and omega1). Everything
runs in the CUDA library; tensors only carry values in and out.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lbkm


class DetonationObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho0, S, Q, omega1, setup):
        p = dict(setup["params"])
        s = lbkm.Solver(nx=p["nx"], ny=1, precision=lbkm.F64, gamma=p["gamma"],
                        orbit_kind=p["orbit_kind"], orbit_speed=p["orbit_speed"],
                        orbit_eta=p["orbit_eta"], S=S.detach().double().cpu().numpy(),
                        Q=float(Q), omega1=float(omega1), omega2=0.0, T_ig=p["T_ig"],
                        dx=p["dx"], dy=p["dx"], dt=p["dt"], bc=(p.get("bc_x", 1), 0))
        f = setup["fields"]
        s.init_fields(rho0.detach().double().cpu().numpy().reshape(1, -1), f["ux"], f["uy"],
                      f["T"], f["lam"])
        g = s.grad(setup["rho_target"], setup["steps"], w_mismatch=setup.get("w_mismatch", 1.0),
                   w_tne=setup.get("w_tne", 1.0),
                   checkpoint_every=setup.get("checkpoint_every", 64))
        s.close()
        dev = rho0.device
        ctx.save_for_backward(torch.as_tensor(g["drho0"], device=dev).reshape(rho0.shape),
                              torch.as_tensor(g["dS"], device=dev),
                              torch.tensor(g["dQ"], dtype=torch.float64, device=dev),
                              torch.tensor(g["domega1"], dtype=torch.float64, device=dev))
        return torch.tensor(g["J"], dtype=torch.float64, device=dev)

    @staticmethod
    def backward(ctx, gJ):
        drho0, dS, dQ, dk = ctx.saved_tensors
        return gJ * drho0, gJ * dS, gJ * dQ, gJ * dk, None
