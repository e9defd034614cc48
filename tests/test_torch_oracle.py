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


def test_omega2_forward_and_gradient(oracle_mod):
    """omega2 != 0 takes the general closed form of Eq. (28) (m = n = 1): the forward map
    equals the C oracle's, and dJ/domega2 by reverse mode equals central differences."""
    nx, steps, w2 = 96, 60, 800.0
    c, p, _ = setup(nx, steps)
    m = to.Model1D(nx, gamma=p["gamma"], orbit_kind=p["orbit_kind"],
                   orbit_speed=p["orbit_speed"], orbit_eta=p["orbit_eta"], T_ig=p["T_ig"],
                   dx=p["dx"], dt=p["dt"], omega2=w2)
    q = dict(p, omega2=w2)
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
    assert lam.sum() > np.sum(fl["lam"]) + 1e-3  # the reaction ran

    rho_t = to.to_t(f[:, 0].sum(axis=0) * 1.001)
    args = [to.to_t(fl[k_][0]) for k_ in ("rho", "ux", "uy", "T", "lam")]

    def J(w):
        m.omega2 = w
        return to.objective(m, *args, S, Q, k, steps, rho_t, 1.0)[0]

    w = torch.tensor(w2, dtype=torch.float64, requires_grad=True)
    (g,) = torch.autograd.grad(J(w), w)
    # J moves little with omega2 (omega2 dJ/domega2 is 2.5e-4 of J), so the step is larger than
    # elsewhere to keep J's rounding out of the difference quotient
    h = 1e-4 * w2
    with torch.no_grad():
        Jp, bp = to.record_branches(lambda: J(torch.tensor(w2 + h, dtype=torch.float64)))
        Jm, bm = to.record_branches(lambda: J(torch.tensor(w2 - h, dtype=torch.float64)))
    assert len(bp) == len(bm) and all(torch.equal(x, y) for x, y in zip(bp, bm))
    fd = (float(Jp) - float(Jm)) / (2 * h)
    assert fd != 0.0 and abs(fd - float(g)) <= 1e-6 * abs(fd), (fd, float(g))


def test_restarted_segments_equal_the_c_oracle_run_segment_by_segment(oracle_mod):
    """objective(..., restarts=...) against the C oracle stepped segment by segment from
    the same restart states (here: a run's states rounded to FP32 at every checkpoint):
    J = 1/2 sum (rho_N - rho*)^2 dx + w sum_n sum_x d_n^2 dx dt, the TNE part from the C
    oracle's record of each state (its sums carry dx dy)."""
    nx, steps, ck, w_tne = 64, 30, 8, 0.7
    c, p, m = setup(nx, steps)
    q = dict(p)
    q.pop("nx"), q.pop("ny")
    ob = oracle_mod.Oracle(nx, 1, **q)
    fl = c["fields"]
    r32 = lambda a: np.asarray(a, np.float64).astype(np.float32).astype(np.float64)  # noqa: E731
    f = ob.init(fl["rho"], fl["ux"], fl["uy"], fl["T"])
    lam = np.broadcast_to(fl["lam"], (1, nx)).astype(np.float64)
    dy = q.get("dy") or q["dx"]
    tne, restarts = 0.0, []
    for n in range(steps):
        if n % ck == 0:
            f, lam = r32(f), r32(lam)
            restarts.append((f[:, 0].copy(), lam[0].copy()))
        tne += ob.tne(f, fields=False)[1]["d2_sum"] / dy * q["dt"]
        f, lam = ob.step(f, lam)
    rho_t = 1.0 + 0.01 * np.cos(np.arange(nx))
    J_c = 0.5 * ((f[:, 0].sum(axis=0) - rho_t) ** 2).sum() * q["dx"] + w_tne * tne
    S, Q, k = to.to_t(p["S"]), torch.tensor(p["Q"]), torch.tensor(p["omega1"])
    args = [to.to_t(fl[k_][0]) for k_ in ("rho", "ux", "uy", "T", "lam")]
    J_t, _, _ = to.objective(m, *args, S, Q, k, steps, to.to_t(rho_t), w_tne,
                             checkpoint_every=ck, restarts=restarts)
    J_64, _, _ = to.objective(m, *args, S, Q, k, steps, to.to_t(rho_t), w_tne)
    assert abs(float(J_t) - J_c) <= 1e-12 * abs(J_c), (float(J_t), J_c)
    assert float(J_t) != float(J_64)  # the restarts are there


def test_restarts_at_the_trajectory_s_own_states_change_nothing():
    """Restarting each segment from the state the previous one reached leaves J and every
    gradient bit for bit as they are: the restarts only replace values."""
    nx, steps, ck = 64, 24, 8
    c, p, m = setup(nx, steps)
    fl = c["fields"]
    rho_t = to.to_t(1.0 + 0.01 * np.cos(np.arange(nx)))
    S0, Q0, k0 = to.to_t(p["S"]), torch.tensor(p["Q"]), torch.tensor(p["omega1"])
    with torch.no_grad():
        f = m.init(*[to.to_t(fl[k_][0]) for k_ in ("rho", "ux", "uy", "T")])
        lam = to.to_t(fl["lam"][0])
        restarts = []
        for n in range(steps):
            if n % ck == 0:
                restarts.append((f.clone(), lam.clone()))
            f, lam, _ = m.step(f, lam, S0, Q0, k0)

    def run(rs):
        S = S0.clone().requires_grad_(True)
        rho0 = to.to_t(fl["rho"][0]).requires_grad_(True)
        J = to.objective(m, rho0, *[to.to_t(fl[k_][0]) for k_ in ("ux", "uy", "T", "lam")],
                         S, Q0, k0, steps, rho_t, 1.0, checkpoint_every=ck, restarts=rs)[0]
        J.backward()
        return float(J), S.grad.numpy(), rho0.grad.numpy()

    a, b = run(None), run(restarts)
    assert a[0] == b[0]
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_periodic_forward_matches_c_oracle(oracle_mod):
    """The periodic ends (images of the far cells as ghosts) against the C oracle with
    bc_x = periodic, on a state whose fronts cross both ends."""
    nx, steps = 96, 80
    c, p, _ = setup(nx, steps, omega1=2e4)
    m = to.Model1D(nx, gamma=p["gamma"], orbit_kind=p["orbit_kind"],
                   orbit_speed=p["orbit_speed"], orbit_eta=p["orbit_eta"], T_ig=p["T_ig"],
                   dx=p["dx"], dt=p["dt"], periodic=True)
    q = dict(p, bc_x=0)
    q.pop("nx"), q.pop("ny")
    ob = oracle_mod.Oracle(nx, 1, **q)
    fl = c["fields"]
    # the driver straddles the end: the state is shifted by half the grid
    fl = {k: np.roll(np.asarray(v, float), nx // 2 + 10, axis=-1) for k, v in fl.items()}
    f, lam = ob.run(ob.init(fl["rho"], fl["ux"], fl["uy"], fl["T"]), fl["lam"], steps)
    ft = m.init(*[to.to_t(fl[k][0]) for k in ("rho", "ux", "uy", "T")])
    lt = to.to_t(fl["lam"][0])
    S, Q, k = to.to_t(p["S"]), torch.tensor(p["Q"]), torch.tensor(p["omega1"])
    for _ in range(steps):
        ft, lt, _ = m.step(ft, lt, S, Q, k)
    assert np.abs(ft.numpy() - f[:, 0]).max() <= 1e-13 * np.abs(f).max()
    assert np.abs(lt.numpy() - lam[0]).max() <= 1e-13
