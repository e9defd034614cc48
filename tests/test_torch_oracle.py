"""Pins of the differentiable FP64 reference (oracle/torch_oracle.py): its forward map
equals the C oracle's, and its reverse-mode gradient equals central finite
differences wherever the + and - runs take the same branches (ignition switch,
minmod choices, upwind side, clamp)."""
import numpy as np
import pytest
import torch

import lbkm_inputs as li
from oracle import torch_oracle as to


def setup(nx=96, steps=60, omega1=2e3):
    c = li.detonation(nx=nx, steps=steps, driver=16, omega1=omega1)
    p = dict(c["params"])
    m = to.Model1D(nx, gamma=p["gamma"], orbit_kind=p["orbit_kind"],
                   orbit_speed=p["orbit_speed"], orbit_eta=p["orbit_eta"], T_ig=p["T_ig"],
                   dx=p["dx"], dt=p["dt"])
    return c, p, m


def test_forward_matches_c_oracle(oracle_mod):
    nx, steps = 128, 80
    c, p, m = setup(nx, steps, omega1=2e4)
    q = dict(p)
    q.pop("nx"), q.pop("ny")
    ob = oracle_mod.Oracle(nx, 1, **q)
    fl = c["fields"]
    f, lam = ob.run(ob.init(fl["rho"], fl["ux"], fl["uy"], fl["T"]), fl["lam"], steps)
    ft = m.init(*[to.to_t(fl[k][0]) for k in ("rho", "ux", "uy", "T")])
    lt = to.to_t(fl["lam"][0])
    S, Q, k = to.to_t(p["S"]), torch.tensor(p["Q"]), torch.tensor(p["omega1"])
    for _ in range(steps):
        ft, lt, _ = m.step(ft, lt, S, Q, k)
    assert np.abs(ft.numpy() - f[:, 0]).max() <= 1e-13 * np.abs(f).max()
    assert np.abs(lt.numpy() - lam[0]).max() <= 1e-13


def _J(m, c, p, theta, rho_t, w_tne, steps):
    fl = c["fields"]
    S = theta[:16]
    return to.objective(m, theta[18:], to.to_t(fl["ux"][0]), to.to_t(fl["uy"][0]),
                        to.to_t(fl["T"][0]), to.to_t(fl["lam"][0]), S, theta[16], theta[17],
                        steps, rho_t, w_tne)[0]


def test_gradient_matches_central_differences():
    nx, steps = 96, 60
    c, p, m = setup(nx, steps)
    fl = c["fields"]
    theta0 = torch.cat([to.to_t(p["S"]), torch.tensor([p["Q"], p["omega1"]], dtype=torch.float64),
                        to.to_t(fl["rho"][0])])
    # target: the same run with perturbed rates and heat release
    rng = np.random.default_rng(5)
    th_t = theta0.clone()
    th_t[4:16] *= torch.as_tensor(1 + 0.05 * rng.standard_normal(12))
    th_t[16] *= 1.05
    with torch.no_grad():
        f = m.init(th_t[18:], *[to.to_t(fl[k][0]) for k in ("ux", "uy", "T")])
        lam = to.to_t(fl["lam"][0])
        for _ in range(steps):
            f, lam, _ = m.step(f, lam, th_t[:16], th_t[16], th_t[17])
        rho_t = m.M[0] @ f
    w_tne = 1.0
    th = theta0.clone().requires_grad_(True)
    J = _J(m, c, p, th, rho_t, w_tne, steps)
    (g,) = torch.autograd.grad(J, th)
    checked = 0
    for idx in [4, 5, 6, 7, 8, 11, 15, 16, 17, 18 + 3, 18 + 20, 18 + 40]:
        h = 1e-6 * abs(float(theta0[idx]))
        tp, tm = theta0.clone(), theta0.clone()
        tp[idx] += h
        tm[idx] -= h
        with torch.no_grad():
            Jp, bp = to.record_branches(lambda: _J(m, c, p, tp, rho_t, w_tne, steps))
            Jm, bm = to.record_branches(lambda: _J(m, c, p, tm, rho_t, w_tne, steps))
        if len(bp) != len(bm) or any(not torch.equal(x, y) for x, y in zip(bp, bm)):
            continue  # a branch flipped between the two runs: no derivative to compare
        fd = (float(Jp) - float(Jm)) / (2 * h)
        assert abs(fd - float(g[idx])) <= 1e-6 * abs(fd) + 1e-12 * abs(float(J)), (idx, fd, g[idx])
        checked += 1
    assert checked >= 8
