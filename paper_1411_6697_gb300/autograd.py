"""torch.autograd.Function over the adjoint of the fused step (lbkm_grad).

``detonation_objective(rho0, S, Q, omega1, setup, omega2=None)`` runs the 1-D model from
the equilibrium start (rho0, u0, T0, lambda0) for ``setup["steps"]`` steps and returns
J = w_mismatch/2 sum (rho_N - rho*)^2 dx + w_tne sum_n sum_x d_n^2 dx dt (Sec. VI,
Eqs. (90)-(91)). When gradients are recorded and an argument requires one, it goes
through ``DetonationObjective``, whose forward takes J and every gradient from one
adjoint sweep (lbkm_grad) and whose backward scales them: gradients of J with respect
to rho0, the 16 rates S, Q, omega1 and omega2 (Eq. (28)). Otherwise it takes J alone
(lbkm_objective_value: the run without the reverse sweep). ``setup["precision"]`` is
"f64" (default) or "f32": the FP32 run, with J and its derivative taken along FP64
segments restarted from its states every ``setup["checkpoint_every"]`` steps.
Everything runs in the CUDA library; tensors only carry values in and out.
"""
from __future__ import annotations

import torch

from . import lbkm


def _solver(rho0, S, Q, omega1, omega2, setup):
    p = dict(setup["params"])
    prec = {"f64": lbkm.F64, "f32": lbkm.F32}[setup.get("precision", "f64")]
    s = lbkm.Solver(nx=p["nx"], ny=1, precision=prec, gamma=p["gamma"],
                    orbit_kind=p["orbit_kind"], orbit_speed=p["orbit_speed"],
                    orbit_eta=p["orbit_eta"], S=S.detach().double().cpu().numpy(),
                    Q=float(Q), omega1=float(omega1),
                    omega2=0.0 if omega2 is None else float(omega2), T_ig=p["T_ig"],
                    dx=p["dx"], dy=p["dx"], dt=p["dt"], bc=(p.get("bc_x", 1), 0))
    f = setup["fields"]
    s.init_fields(rho0.detach().double().cpu().numpy().reshape(1, -1), f["ux"], f["uy"],
                  f["T"], f["lam"])
    return s


def _objective_args(setup):
    return dict(w_mismatch=setup.get("w_mismatch", 1.0), w_tne=setup.get("w_tne", 1.0),
                checkpoint_every=setup.get("checkpoint_every", 64))


class DetonationObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho0, S, Q, omega1, setup, omega2=None):
        s = _solver(rho0, S, Q, omega1, omega2, setup)
        try:
            g = s.grad(setup["rho_target"], setup["steps"], **_objective_args(setup))
        finally:
            s.close()
        dev = rho0.device
        ctx.save_for_backward(torch.as_tensor(g["drho0"], device=dev).reshape(rho0.shape),
                              torch.as_tensor(g["dS"], device=dev),
                              torch.tensor(g["dQ"], dtype=torch.float64, device=dev),
                              torch.tensor(g["domega1"], dtype=torch.float64, device=dev),
                              torch.tensor(g["domega2"], dtype=torch.float64, device=dev))
        return torch.tensor(g["J"], dtype=torch.float64, device=dev)

    @staticmethod
    def backward(ctx, gJ):
        drho0, dS, dQ, dk1, dk2 = ctx.saved_tensors
        need = ctx.needs_input_grad
        return (gJ * drho0, gJ * dS, gJ * dQ, gJ * dk1, None,
                gJ * dk2 if len(need) > 5 and need[5] else None)


def detonation_objective(rho0, S, Q, omega1, setup, omega2=None):
    """J of the run (a 0-d float64 tensor on rho0's device); differentiable in rho0, S, Q,
    omega1 and omega2 (a tensor, or None for omega2 = 0 held fixed)."""
    args = [t for t in (rho0, S, Q, omega1, omega2) if isinstance(t, torch.Tensor)]
    if torch.is_grad_enabled() and any(t.requires_grad for t in args):
        if omega2 is None:
            return DetonationObjective.apply(rho0, S, Q, omega1, setup)
        return DetonationObjective.apply(rho0, S, Q, omega1, setup, omega2)
    s = _solver(rho0, S, Q, omega1, omega2, setup)
    try:
        J = s.objective(setup["rho_target"], setup["steps"], **_objective_args(setup))["J"]
    finally:
        s.close()
    return torch.tensor(J, dtype=torch.float64, device=rho0.device)
