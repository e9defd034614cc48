"""The CUDA discrete adjoint (lbkm_grad) against the FP64 reverse-mode oracle
(oracle/torch_oracle.py, itself pinned to the C oracle and to central differences):
objective value and gradients with respect to S, Q, omega1 and the initial density."""
import numpy as np
import pytest
import torch

import lbkm_inputs as li
from oracle import torch_oracle as to
from paper_1411_6697_gb300 import lbkm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    assert torch.cuda.is_available(), "the -m gpu tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()


def problem(nx, steps, omega1, driver):
    # the ripple keeps the minmod branches of the f_i away from rounding-level
    # differences; on flat stretches the gradient would depend on how each side rounds
    # (without it the oracle's own drho0 near the boundary differs by ~10 % between an
    # x86 and an Arm host)
    c = li.detonation(nx=nx, steps=steps, driver=driver, omega1=omega1, ripple=1e-3)
    p = dict(c["params"])
    m = to.Model1D(nx, gamma=p["gamma"], orbit_kind=p["orbit_kind"],
                   orbit_speed=p["orbit_speed"], orbit_eta=p["orbit_eta"], T_ig=p["T_ig"],
                   dx=p["dx"], dt=p["dt"])
    fl = c["fields"]
    # target: the run with perturbed rates and heat release (as the adjoint workload)
    rng = np.random.default_rng(li.SEED_BASE + 5)
    S_t = np.asarray(p["S"]) * (1 + 0.05 * rng.standard_normal(16))
    with torch.no_grad():
        f = m.init(*[to.to_t(fl[k][0]) for k in ("rho", "ux", "uy", "T")])
        lam = to.to_t(fl["lam"][0])
        for _ in range(steps):
            f, lam, _ = m.step(f, lam, to.to_t(S_t), torch.tensor(p["Q"] * 1.05),
                               torch.tensor(p["omega1"]))
        rho_t = (m.M[0] @ f).numpy()
    return c, p, m, rho_t


def oracle_grad(c, p, m, rho_t, steps, w_tne, ck=0):
    fl = c["fields"]
    rho0 = to.to_t(fl["rho"][0]).requires_grad_(True)
    S = to.to_t(p["S"]).requires_grad_(True)
    Q = torch.tensor(p["Q"], dtype=torch.float64, requires_grad=True)
    k = torch.tensor(p["omega1"], dtype=torch.float64, requires_grad=True)
    J, mis, tne = to.objective(m, rho0, to.to_t(fl["ux"][0]), to.to_t(fl["uy"][0]),
                               to.to_t(fl["T"][0]), to.to_t(fl["lam"][0]), S, Q, k, steps,
                               to.to_t(rho_t), w_tne, checkpoint_every=ck)
    J.backward()
    return dict(J=float(J), J_mismatch=float(mis), dS=S.grad.numpy(), dQ=float(Q.grad),
                domega1=float(k.grad), drho0=rho0.grad.numpy())


def gpu_grad(c, p, rho_t, steps, w_tne, ck):
    fl = c["fields"]
    s = lbkm.Solver(nx=p["nx"], ny=1, precision=lbkm.F64, gamma=p["gamma"],
                    orbit_kind=p["orbit_kind"], orbit_speed=p["orbit_speed"],
                    orbit_eta=p["orbit_eta"], S=p["S"], Q=p["Q"], omega1=p["omega1"],
                    T_ig=p["T_ig"], dx=p["dx"], dy=p["dx"], dt=p["dt"], bc=(1, 0))
    s.init_fields(fl["rho"], fl["ux"], fl["uy"], fl["T"], fl["lam"])
    before = s.get_state()
    g = s.grad(rho_t, steps, w_tne=w_tne, checkpoint_every=ck)
    assert np.array_equal(s.get_state(), before)  # the handle's state is untouched
    return g


def compare(g, r, tol, tol_rho0=None):
    assert abs(g["J"] - r["J"]) <= tol * abs(r["J"])
    assert abs(g["J_mismatch"] - r["J_mismatch"]) <= tol * abs(r["J_mismatch"])
    sc = np.abs(r["dS"][4:]).max()
    assert np.abs(g["dS"][4:] - r["dS"][4:]).max() <= tol * sc, (g["dS"], r["dS"])
    assert np.all(g["dS"][:4] == 0) and np.abs(r["dS"][:4]).max() == 0.0
    assert abs(g["dQ"] - r["dQ"]) <= tol * abs(r["dQ"])
    assert abs(g["domega1"] - r["domega1"]) <= tol * abs(r["domega1"])
    t0 = tol if tol_rho0 is None else tol_rho0
    assert np.abs(g["drho0"] - r["drho0"]).max() <= t0 * np.abs(r["drho0"]).max()


@pytest.mark.parametrize("ck", [16, 7, 60])
def test_adjoint_matches_reverse_mode_oracle_small(ck):
    nx, steps = 96, 60
    c, p, m, rho_t = problem(nx, steps, omega1=2e3, driver=16)
    r = oracle_grad(c, p, m, rho_t, steps, w_tne=1.0)
    g = gpu_grad(c, p, rho_t, steps, w_tne=1.0, ck=ck)
    compare(g, r, 1e-9)


@pytest.mark.slow
def test_adjoint_full_config_size():
    """8192 cells, 4000 steps, checkpoints every 64, config-2 parameters (k = 2e4)."""
    nx, steps = 8192, 4000
    c, p, m, rho_t = problem(nx, steps, omega1=2e4, driver=50)
    r = oracle_grad(c, p, m, rho_t, steps, w_tne=1.0, ck=64)
    g = gpu_grad(c, p, rho_t, steps, w_tne=1.0, ck=64)
    # behind the front lambda sits within a few ulp of 1, so the minmod branches of
    # u.grad(lambda) there are decided by rounding: flipping every such branch whose
    # arguments are below 1e-15 moves the oracle's own drho0 by 2.9e-7 of its maximum
    # (and J, dS, dQ, domega1 by < 1e-11), hence the wider elementwise bound on drho0
    compare(g, r, 1e-7, tol_rho0=2e-6)


def test_autograd_function_backward():
    from paper_1411_6697_gb300.autograd import DetonationObjective
    nx, steps = 64, 40
    c, p, m, rho_t = problem(nx, steps, omega1=2e3, driver=12)
    setup = dict(params=p, fields=c["fields"], rho_target=rho_t, steps=steps, w_tne=1.0,
                 checkpoint_every=16)
    rho0 = torch.tensor(c["fields"]["rho"][0], dtype=torch.float64, requires_grad=True)
    S = torch.tensor(p["S"], dtype=torch.float64, requires_grad=True)
    Q = torch.tensor(p["Q"], dtype=torch.float64, requires_grad=True)
    k = torch.tensor(p["omega1"], dtype=torch.float64, requires_grad=True)
    J = DetonationObjective.apply(rho0, S, Q, k, setup)
    (2.0 * J).backward()
    r = oracle_grad(c, p, m, rho_t, steps, w_tne=1.0)
    assert abs(float(J) - r["J"]) <= 1e-9 * abs(r["J"])
    assert np.allclose(rho0.grad.numpy(), 2 * r["drho0"], rtol=0,
                       atol=1e-9 * np.abs(r["drho0"]).max())
    assert np.allclose(S.grad.numpy()[4:], 2 * r["dS"][4:], rtol=0,
                       atol=1e-9 * np.abs(r["dS"]).max())
    assert abs(float(Q.grad) - 2 * r["dQ"]) <= 1e-9 * abs(r["dQ"])
