"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties the oracle to something other than itself: a quadrature of the
continuous Maxwellian, a library ODE solver or linear solve, an independent
brute-force formulation, conservation laws, the exact Euler Riemann solution,
Chapman-Jouguet theory, the shear viscosity of the Chapman-Enskog analysis, and
values printed in the paper (tests/golden).
"""
import os

import numpy as np
import pytest

import brute_force as bf
import exact_riemann as er
import lbkm_inputs as li

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def make(oracle_mod, nx, ny, **kw):
    base = dict(gamma=1.4, **li.DEFAULT_ORBITS, S=1e5)
    base.update(kw)
    return oracle_mod.Oracle(nx, ny, **base)


def read_golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


# ---------------------------------------------------------------- M, M^-1
def test_moment_matrix_inverse(oracle_mod):
    ob = make(oracle_mod, 4, 1)
    assert np.abs(ob.M @ ob.Minv - np.eye(16)).max() < 1e-13
    # independent inverse from a library routine, and M from moment functions
    vx, vy, eta = bf.velocity_set(*[li.DEFAULT_ORBITS[k] for k in
                                    ("orbit_kind", "orbit_speed", "orbit_eta")])
    M2 = bf.moment_matrix(vx, vy, eta)
    assert np.allclose(M2, ob.M, rtol=1e-14, atol=0)
    Minv2 = np.linalg.inv(M2)
    assert np.abs(Minv2 - ob.Minv).max() < 1e-12 * np.abs(Minv2).max()


def test_two_ring_cut_of_d2v24_is_singular(oracle_mod):
    """The paper's first two rings (axis and diagonal sharing one speed and eta, Sec. II)
    give a rank-14 M under rows m1..m16: the 16-velocity model needs 4 orbits."""
    with pytest.raises(ValueError):
        make(oracle_mod, 4, 1, orbit_kind=(0, 1, 0, 1), orbit_speed=(2.7, 2.7, 2.2, 2.2),
             orbit_eta=(5.0, 5.0, 3.0, 3.0))


# ---------------------------------------------------------------- f^eq
@pytest.mark.parametrize("seed", range(5))
def test_feq_moments_match_maxwellian_quadrature(oracle_mod, seed):
    """f_hat^eq (list after Eq. (16), entries 14 and 16 per Eq. (11)) equals the moments
    of the continuous Maxwellian Eq. (21), computed by Gauss-Hermite quadrature."""
    rng = np.random.default_rng(seed)
    rho, ux, uy, T = rng.uniform(0.2, 3), rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0.3, 3)
    gamma = rng.choice([1.4, 1.5, 5 / 3 - 1e-9 + 1e-9, 1.25])
    ob = make(oracle_mod, 4, 1, gamma=gamma)
    I = ob.p.I
    q = bf.maxwellian_moments(rho, ux, uy, T, I)
    got = ob.feq_moments(rho, ux, uy, T)
    assert np.allclose(got, q, rtol=1e-12, atol=1e-12 * np.abs(q).max())


def test_feq_14_16_carry_factor_T(oracle_mod):
    """The printed f_hat^eq_14 drops a factor T that Eq. (11) carries; the quadrature
    decides: at T != 1 only the Eq. (11) form matches."""
    ob = make(oracle_mod, 4, 1)
    rho, ux, uy, T, I = 1.3, 0.4, -0.2, 2.0, ob.p.I
    q = bf.maxwellian_moments(rho, ux, uy, T, I)
    u2 = ux * ux + uy * uy
    printed = rho * ((2 + I + 2) * T + u2) + rho * ux * ux * ((2 + I + 4) * T + u2)
    assert abs(ob.feq_moments(rho, ux, uy, T)[13] - q[13]) < 1e-12 * abs(q[13])
    assert abs(printed - q[13]) > 1e-2 * abs(q[13])


@pytest.mark.parametrize("seed", range(4))
def test_dfeq_dT_matches_eq22_quadrature(oracle_mod, seed):
    """d f_hat^eq/dT equals the moments of df^eq/dT as given by Eq. (22)."""
    rng = np.random.default_rng(100 + seed)
    rho, ux, uy, T = rng.uniform(0.2, 3), rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0.3, 3)
    ob = make(oracle_mod, 4, 1)
    q = bf.maxwellian_moments(rho, ux, uy, T, ob.p.I, dT=True)
    got = ob.dfeq_dT(rho, ux, uy, T)
    assert np.allclose(got, q, rtol=1e-11, atol=1e-11 * np.abs(q).max())


def test_chemical_term_matches_sec3_values(oracle_mod):
    """C_hat_k = (d f_hat^eq_k/dT) 2 Q lambda'/(D+I) reproduces the values the paper states
    for k = 1..9 in Sec. III: C1=C2=C3=C6=0, C4=2 rho lambda' Q, C5=C7=C4/(D+I),
    C8 = C4 u_x (D+I+2)/(D+I), C9 = C4 u_y (D+I+2)/(D+I)."""
    ob = make(oracle_mod, 4, 1, gamma=1.5)
    rho, ux, uy, T, Q, lp = 1.2, 0.3, -0.4, 1.7, 0.8, 3.1
    DI = 2 + ob.p.I
    C = ob.dfeq_dT(rho, ux, uy, T) * 2 * Q * lp / DI
    C4 = 2 * rho * lp * Q
    want = [0, 0, 0, C4, C4 / DI, 0, C4 / DI, C4 * ux * (DI + 2) / DI, C4 * uy * (DI + 2) / DI]
    assert np.allclose(C[:9], want, rtol=1e-14, atol=1e-14)


# ---------------------------------------------------------------- reaction
@pytest.mark.parametrize("lam,a,b", [(0.0, 4e4, 0.0), (0.3, 1e3, 0.0), (0.7, 2e4, 5e3),
                                     (0.05, 100.0, 900.0), (1.0, 1e4, 1e4)])
def test_reaction_increment_vs_ode_solver(oracle_mod, lam, a, b):
    """Exact time integration of Eq. (28) (m = n = 1) against a high-order ODE solver."""
    from scipy.integrate import solve_ivp
    dt = 2e-6 * 7
    sol = solve_ivp(lambda _, z: (1 - z) * (a + b * z), (0, dt), [lam], method="DOP853",
                    rtol=1e-13, atol=1e-16)
    assert abs(oracle_mod.reaction_increment(lam, a, b, dt) - (sol.y[0, -1] - lam)) < 1e-12


# ---------------------------------------------------------------- step invariants
def test_uniform_equilibrium_is_fixed(oracle_mod):
    """A uniform equilibrium with no reaction stays put: advection vanishes identically
    and f_hat = f_hat^eq makes the collision zero."""
    for T0, Q in ((1.0, 1.0), (1.3, 0.0)):  # below ignition / no heat release
        ob = make(oracle_mod, 6, 5, Q=Q, omega1=2e4, bc_x=0, bc_y=0,
                  S=np.linspace(1e4, 1e5, 16))
        f0 = ob.init(1.2, 0.3, -0.2, T0)
        f, lam = ob.run(f0, 0.25, 100)
        assert np.abs(f - f0).max() < 1e-13 * np.abs(f0).max()
        if T0 < 1.1:
            assert np.all(lam == 0.25)  # below ignition nothing reacts
        else:
            assert np.all(lam > 0.25)  # Q = 0: lambda burns but releases no heat


def test_collision_conserves_and_heats(oracle_mod):
    """On a uniform non-equilibrium state (no advection) rows 1-3 of M (f_new - f) vanish
    and row 4 gains 2 rho Q dlambda: Omega_hat_1..3 = 0, Omega_hat_4 = C_hat_4 (Sec. III)."""
    rng = np.random.default_rng(7)
    ob = make(oracle_mod, 3, 2, Q=1.0, omega1=2e4, omega2=3e3, T_ig=1.1, bc_x=0, bc_y=0,
              S=rng.uniform(1e3, 1e5, 16), dt=2e-6)
    feq = ob.init(1.1, 0.2, 0.1, 1.5)
    f = feq + 1e-3 * rng.standard_normal(16)[:, None, None] * np.abs(feq)
    lam0 = 0.4
    f1, lam1 = ob.step(f, lam0)
    dm = np.einsum("ki,iyx->kyx", ob.M, f1 - f)
    rho = ob.macros(f)["rho"]
    scale = np.abs(np.einsum("ki,iyx->kyx", np.abs(ob.M), np.abs(f))).max()
    assert np.abs(dm[:3]).max() < 1e-13 * scale
    assert lam1[0, 0] > lam0
    assert np.allclose(dm[3], 2 * rho * ob.p.Q * (lam1 - lam0), rtol=1e-10)


def test_conservation_periodic_2d(oracle_mod):
    """Periodic 2-D flow without reaction: total mass, momentum and energy are constant
    (NND fluxes telescope; the collision conserves rows 1-4)."""
    rng = np.random.default_rng(11)
    nx, ny = 16, 12
    x = np.arange(nx) / nx
    y = np.arange(ny)[:, None] / ny
    rho = 1 + 0.2 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    ux = 0.3 * np.cos(2 * np.pi * y) + 0 * x
    uy = 0.2 * np.sin(2 * np.pi * x) + 0 * y
    T = 1 + 0.1 * np.cos(2 * np.pi * (x + y))
    ob = make(oracle_mod, nx, ny, bc_x=0, bc_y=0, S=rng.uniform(1e3, 1e4, 16), dx=1e-2,
              dt=1e-4)
    f0 = ob.init(rho, ux, uy, T)
    f, _ = ob.run(f0, 0.0, 50)
    tot0 = np.einsum("ki,iyx->k", ob.M[:4], f0)
    tot = np.einsum("ki,iyx->k", ob.M[:4], f)
    assert np.all(np.abs(tot - tot0) < 1e-12 * np.abs(np.einsum("ki,iyx->k", np.abs(ob.M[:4]),
                                                                   np.abs(f0))))
    assert np.abs(f - f0).max() > 1e-4  # the flow did evolve


def test_heat_release_equals_Q_rho_dlambda(oracle_mod):
    """With reaction (uniform lambda, so no lambda advection): total energy grows by
    Q sum(rho dlambda) (Eq. (18)), momentum and mass stay constant."""
    nx = 10
    x = np.arange(nx) / nx
    ob = make(oracle_mod, nx, 1, bc_x=0, Q=1.0, omega1=2e4, T_ig=1.1, dx=1e-3, dt=2e-6)
    rho = 1 + 0.1 * np.sin(2 * np.pi * x)[None, :]
    f0 = ob.init(rho, 0.1 * np.cos(2 * np.pi * x)[None, :], 0.0, 1.3)
    f1, l1 = ob.step(f0, 0.2)
    E0 = 0.5 * np.einsum("i,iyx->", ob.M[3], f0)
    E1 = 0.5 * np.einsum("i,iyx->", ob.M[3], f1)
    gain = ob.p.Q * np.sum(ob.macros(f0)["rho"] * (l1 - 0.2))
    assert gain > 0
    assert abs((E1 - E0) - gain) < 1e-12 * abs(E0)


def test_S1_to_S4_have_no_influence(oracle_mod):
    """R_1..R_4 do not change the evolution (Sec. III)."""
    rng = np.random.default_rng(3)
    S = rng.uniform(1e3, 1e5, 16)
    S2 = S.copy()
    S2[:4] = [1.0, 7.0, 3e9, 0.5]
    c = li.detonation(nx=64, driver=20)
    outs = []
    for s in (S, S2):
        ob = make(oracle_mod, 64, 1, S=s, Q=1.0, omega1=2e4, dx=1e-4, dt=2e-6)
        fl = c["fields"]
        f = ob.init(fl["rho"], fl["ux"], fl["uy"], fl["T"])
        outs.append(ob.run(f, fl["lam"], 30))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_bgk_limit_matches_velocity_space_srt(oracle_mod):
    """With all R_k equal, A_hat vanishes and the step is the SRT form Eq. (87):
    f_new = f + dt(-(f - M^-1 f_hat^eq)/tau - v.grad f), checked against the
    independent velocity-space formulation."""
    nx, ny = 6, 5
    rng = np.random.default_rng(5)
    cfg = dict(li.DEFAULT_ORBITS, gamma=1.4, S=np.full(16, 3e4), Q=0.0, omega1=0.0,
               omega2=0.0, T_ig=1.1, dx=1e-3, dy=1e-3, dt=1e-5, bc_x=0, bc_y=0)
    ob = oracle_mod.Oracle(nx, ny, **{k: v for k, v in cfg.items()})
    x = np.arange(nx) / nx
    y = np.arange(ny)[:, None] / ny
    f = ob.init(1 + 0.1 * np.sin(2 * np.pi * x) + 0 * y, 0.2 * np.cos(2 * np.pi * y) + 0 * x,
                -0.1 + 0 * (x + y), 1.1 + 0.05 * np.cos(2 * np.pi * (x - y)))
    f = f * (1 + 1e-3 * rng.standard_normal(f.shape))
    lam = rng.uniform(0, 0.5, (ny, nx))
    fo, lo = ob.step(f, lam)
    fb, lb = bf.step(cfg, f, lam)
    assert np.abs(fo - fb).max() < 1e-12 * np.abs(f).max()
    assert np.abs(lo - lb).max() < 1e-13


@pytest.mark.parametrize("nx,ny,bc_x,bc_y", [(8, 1, 1, 0), (4, 2, 0, 0), (5, 3, 1, 1)])
def test_brute_force_small_grids(oracle_mod, nx, ny, bc_x, bc_y):
    """Oracle vs the naive independent formulation for 10 steps on tiny grids, with
    reaction (both Cochran terms), unequal rates (A_hat active) and 2-D gradients."""
    rng = np.random.default_rng(nx * 100 + ny)
    cfg = dict(li.DEFAULT_ORBITS, gamma=1.4, S=rng.uniform(2e3, 1e5, 16), Q=1.0,
               omega1=2e3, omega2=500.0, T_ig=1.1, dx=1e-3, dy=1e-3, dt=1e-5,
               bc_x=bc_x, bc_y=bc_y)
    ob = oracle_mod.Oracle(nx, ny, **cfg)
    x = np.arange(nx) / nx
    y = np.arange(ny)[:, None] / ny
    rho = 1 + 0.1 * np.sin(2 * np.pi * x) + 0.05 * np.cos(2 * np.pi * y)
    ux = 0.2 * np.cos(2 * np.pi * x) + 0.05 * np.sin(2 * np.pi * y)
    uy = -0.1 + 0.05 * np.sin(2 * np.pi * (x + y))
    T = np.where(x < 0.5, 1.35, 0.95) + 0.02 * np.cos(2 * np.pi * y)
    f = bf.equilibrium(cfg, rho, ux, uy, T)
    f = f * (1 + 2e-3 * rng.standard_normal(f.shape))
    lam = rng.uniform(0, 0.8, (ny, nx))
    fo, lo, fb, lb = f, lam, f, lam
    for _ in range(10):
        fo, lo = ob.step(fo, lo)
        fb, lb = bf.step(cfg, fb, lb)
    assert np.abs(fo - fb).max() < 1e-11 * np.abs(f).max()
    assert np.abs(lo - lb).max() < 1e-12
    # TNE: Delta_k = M f - f_hat^eq with f^eq from quadrature
    delta, rec = ob.tne(fo)
    m = ob.macros(fo)
    for (yy, xx) in [(0, 0), (ny - 1, nx - 1)]:
        fh = ob.M @ fo[:, yy, xx]
        q = bf.maxwellian_moments(m["rho"][yy, xx], m["ux"][yy, xx], m["uy"][yy, xx],
                                  m["T"][yy, xx], ob.p.I)
        assert np.allclose(delta[4:, yy, xx], (fh - q)[4:], atol=1e-12 * np.abs(fh).max())
        assert np.all(delta[:4, yy, xx] == 0)


@pytest.mark.parametrize("nv", [16, 24])
def test_tne_grid_record_matches_independent_sums(oracle_mod, nv):
    """The oracle's grid-wide TNE record (Sec. VI, Eqs. (90)-(91)) against the same record
    rebuilt by the brute-force formulation: Delta_k from its own moment functions and the
    quadrature Maxwellian, sums of Delta_k, |Delta_k|, d and d^2 weighted by dx dy,
    unweighted min and max. Unequal dx and dy, so a missing or squared cell area, an
    unweighted sum or a weighted extremum all fail; a state driven off equilibrium by a few
    reactive steps, so every Delta_k has both signs."""
    nx, ny = 7, 5
    rng = np.random.default_rng(90 + nv)
    orbits = li.DEFAULT_ORBITS if nv == 16 else li.d2v24_orbits(*li.D2V24_DETONATION_V)
    cfg = dict(orbits, gamma=1.4, S=rng.uniform(2e3, 1e5, nv), Q=1.0, omega1=2e3,
               omega2=0.0, T_ig=1.0, dx=1e-3, dy=2.5e-3, dt=1e-5, bc_x=0, bc_y=0)
    ob = oracle_mod.Oracle(nx, ny, **cfg)
    x = np.arange(nx) / nx
    y = np.arange(ny)[:, None] / ny
    rho = 1 + 0.1 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    ux = 0.2 * np.cos(2 * np.pi * (x + y))
    uy = 0.1 * np.sin(2 * np.pi * y) - 0.05
    T = 1.1 + 0.1 * np.sin(2 * np.pi * (x - y))
    rho, ux, uy, T = (np.broadcast_to(a, (ny, nx)) for a in (rho, ux, uy, T))
    f = bf.equilibrium(cfg, rho, ux, uy, T) * (1 + 3e-3 * rng.standard_normal((nv, ny, nx)))
    f, _ = ob.run(f, rng.uniform(0, 0.5, (ny, nx)), 3)
    delta, rec = ob.tne(f)
    bdelta, brec = bf.tne_record(cfg, f)
    scale = np.abs(bdelta).max()
    assert np.abs(delta - bdelta).max() < 1e-11 * scale
    area = cfg["dx"] * cfg["dy"]
    for key in ("sum", "abs_sum"):
        assert np.allclose(rec[key], brec[key], rtol=0, atol=1e-11 * scale * nx * ny * area)
    for key in ("min", "max"):
        assert np.allclose(rec[key][4:], brec[key][4:], rtol=0, atol=1e-11 * scale)
        assert np.all(rec[key][:4] == 0)
    assert abs(rec["d_sum"] - brec["d_sum"]) < 1e-10 * brec["d_sum"]
    assert abs(rec["d2_sum"] - brec["d2_sum"]) < 1e-10 * brec["d2_sum"]
    # the record is not degenerate: most Delta_k change sign over the grid, extremes
    # apart, d^2 not d
    signs = (brec["min"][4:] < 0) & (brec["max"][4:] > 0)
    assert signs.sum() >= (nv - 4) // 2 and (brec["min"][4:] < brec["max"][4:]).all()
    assert abs(brec["d2_sum"] - brec["d_sum"]) > 0.1 * brec["d_sum"]


# ---------------------------------------------------------------- NND scheme
def test_nnd_conservative_and_non_oscillatory(oracle_mod):
    n = 64
    q = np.where((np.arange(n) > 10) & (np.arange(n) < 30), 1.0, 0.0) + 0.5
    for v in (1.0, -1.0):
        a = q.copy()
        for _ in range(200):
            a = oracle_mod.nnd_advect_1d(v, a, dt=0.5, dx=1.0, bc=0)  # CFL 0.5
            assert a.max() <= 1.5 + 1e-14 and a.min() >= 0.5 - 1e-14
        assert abs(a.sum() - q.sum()) < 1e-11


def test_nnd_second_order_on_smooth_data(oracle_mod):
    """Spatial order of the NND flux at a small CFL number (0.01), where forward Euler's
    O(dt) error is negligible: close to 2, reduced by the limiter at smooth extrema."""
    errs = []
    for n in (64, 128, 256):
        x = (np.arange(n) + 0.5) / n
        a = np.exp(np.sin(2 * np.pi * x))
        dt = 0.01 / n
        steps = int(round(0.25 / dt))
        for _ in range(steps):
            a = oracle_mod.nnd_advect_1d(1.0, a, dt=dt, dx=1.0 / n, bc=0)
        exact = np.exp(np.sin(2 * np.pi * (x - steps * dt)))
        errs.append(np.abs(a - exact).mean())
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0


# ---------------------------------------------------------------- physics
def _run(oracle_mod, cfg):
    p = dict(cfg["params"])
    nx, ny = p.pop("nx"), p.pop("ny")
    ob = oracle_mod.Oracle(nx, ny, **p)
    fl = cfg["fields"]
    f = ob.init(fl["rho"], fl["ux"], fl["uy"], fl["T"])
    f, lam = ob.run(f, fl["lam"], cfg["steps"])
    return ob, f, lam


@pytest.mark.slow
def test_sod_against_exact_riemann_solution(oracle_mod):
    """Sod shock tube (Sec. IV.B) with large R_k: L1 distance to the exact Euler solution
    is small and falls when the grid is refined."""
    errs = []
    for nx, dx, dt in ((200, 2e-3, 1e-5), (400, 1e-3, 1e-5)):  # S dt = 1 < 2 (Euler limit)
        c = li.riemann(nx=nx, steps=int(round(0.05 / dt)), run="A")
        c["params"].update(dx=dx, dt=dt)
        ob, f, _ = _run(oracle_mod, c)
        m = ob.macros(f)
        x = (np.arange(nx) + 0.5) * dx - 0.5 * nx * dx
        r, u, p = er.sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4, x / 0.05)
        errs.append((np.abs(m["rho"][0] - r).mean(), np.abs(m["ux"][0] - u).mean(),
                     np.abs(m["p"][0] - p).mean()))
    assert all(e < 1e-2 for e in errs[1])
    assert all(errs[1][k] < errs[0][k] for k in range(3))


@pytest.mark.slow
@pytest.mark.parametrize("which", ["lax", "sjogreen"])
def test_lax_and_sjogreen_against_exact_riemann_solutions(oracle_mod, which):
    """Lax's shock tube (I = 1) and Sjogreen's double rarefaction (I = 4) of Sec. IV.B,
    run to the paper's end times (t = 0.15 and 0.03) with its grids and collision
    parameters on the 16-velocity table: mean absolute distance of rho, u, p to the
    exact Euler solution. The bounds sit 1.5x (Lax) and 1.15x (Sjogreen) above the
    distances measured; run with gamma = 1.4 instead of the stated I, the Lax distances
    grow tenfold and the Sjogreen rho and u distances by 15 %, past the bounds."""
    c = getattr(li, which)()
    p = c["params"]
    ob, f, _ = _run(oracle_mod, c)
    m = ob.macros(f)
    nx, dx = p["nx"], p["dx"]
    t_end = c["steps"] * p["dt"]
    x = (np.arange(nx) + 0.5) * dx - 0.5 * nx * dx
    (rl, tl, ul), (rr, tr, ur) = c["left"], c["right"]
    r, u, pe = er.sample((rl, ul, rl * tl), (rr, ur, rr * tr), p["gamma"], x / t_end)
    err = (np.abs(m["rho"][0] - r).mean(), np.abs(m["ux"][0] - u).mean(),
           np.abs(m["p"][0] - pe).mean())
    bound = {"lax": (3.7e-3, 3.1e-3, 4.0e-3), "sjogreen": (4.7e-3, 5.4e-3, 1.95e-3)}[which]
    assert all(e < b for e, b in zip(err, bound)), err


@pytest.mark.slow
def test_couette_start_up_against_series_solution(oracle_mod):
    """Couette flow (Sec. IV.D) started from rest, walls by non-equilibrium extrapolation:
    u_x(y, t = 0.5) against the series solution of the start-up problem with nu = T/R_6
    and the walls at y = 0 and y = H = Ny dy. Measured: 1.5 % of u0 at worst, 0.34 % on
    average; with nu off by a factor 2 (R_6 = 4e3) the distances are 12.6 % and 1.9 %."""
    c = li.couette()
    p = c["params"]
    ob, f, _ = _run(oracle_mod, c)
    m = ob.macros(f)
    ny, dy, u0 = p["ny"], p["dx"], c["u0"]
    H, t, nu = ny * dy, c["steps"] * p["dt"], 1.0 / p["S"][5]
    y = (np.arange(ny) + 0.5) * dy
    ua = u0 * y / H + (2.0 / np.pi) * u0 * sum(
        (-1) ** n / n * np.exp(-(n * np.pi) ** 2 * nu * t / H ** 2) * np.sin(n * np.pi * y / H)
        for n in range(1, 400))
    d = np.abs(m["ux"][:, 0] - ua) / u0
    assert d.max() < 0.025 and d.mean() < 0.006, (d.max(), d.mean())
    # the walls conserve nothing in particular, but the channel must stay near rest
    assert np.abs(m["uy"]).max() < 1e-3 * u0 and abs(m["rho"].mean() - 1.0) < 1e-3


def test_time_schemes_converge_at_their_order(oracle_mod):
    """Forward Euler and the two- and three-stage SSP Runge-Kutta schemes built from it, on
    a smooth periodic flow at fixed grid: the difference to a run at dt/16 halves (Euler),
    quarters (SSP-RK2) or falls eightfold (SSP-RK3) when dt halves."""
    nx = 64
    x = (np.arange(nx) + 0.5) / nx
    rho = (1 + 0.05 * np.sin(2 * np.pi * x))[None]
    T = (1 + 0.05 * np.cos(2 * np.pi * x))[None]
    ux = (0.1 * np.sin(4 * np.pi * x))[None]
    z = np.zeros((1, nx))
    S = np.full(16, 200.0)
    S[7:9] = 300.0
    ratios = {}
    for scheme in (0, 1, 2):
        sol = {}
        for k in (1, 2, 4, 16):
            dt = 2e-4 / k
            ob = make(oracle_mod, nx, 1, S=S, dx=1.0 / nx, dt=dt, bc_x=0, time_scheme=scheme)
            f, _ = ob.run(ob.init(rho, ux, z, T), z, int(round(0.05 / dt)))
            sol[k] = f
        e = {k: np.linalg.norm(sol[k] - sol[16]) for k in (1, 2, 4)}
        ratios[scheme] = (e[1] / e[2], e[2] / e[4], e[1])
    assert 1.8 < ratios[0][0] < 2.6 and 1.8 < ratios[0][1] < 2.6, ratios
    assert 3.5 < ratios[1][0] < 4.6 and 3.5 < ratios[1][1] < 4.6, ratios
    assert ratios[1][2] < 1e-2 * ratios[0][2]
    # SSP-RK3: smaller still, but the limiter's kinks in the space operator cap its
    # observed order on this flow (ratios 5.4 then 3.8); its coefficients are pinned
    # exactly by test_time_schemes_follow_their_stability_polynomials
    assert ratios[2][2] < 1e-1 * ratios[1][2]


@pytest.mark.parametrize("scheme", [0, 1, 2])
def test_time_schemes_follow_their_stability_polynomials(oracle_mod, scheme):
    """On a uniform non-equilibrium state (no advection, no reaction, grad u = 0 so
    A_hat = 0) each non-conserved moment relaxes alone, d Delta_k/dt = -R_k Delta_k, and
    one step of a Runge-Kutta scheme multiplies Delta_k by its stability polynomial at
    z = -R_k dt: 1 + z (Euler), 1 + z + z^2/2 (SSP-RK2), 1 + z + z^2/2 + z^3/6 (SSP-RK3)."""
    rng = np.random.default_rng(23)
    S = rng.uniform(1e3, 5e4, 16)
    dt, n = 1e-5, 20
    ob = make(oracle_mod, 3, 2, S=S, dt=dt, bc_x=0, bc_y=0, time_scheme=scheme)
    feq = ob.init(1.1, 0.2, -0.1, 1.3)
    f0 = feq * (1 + 1e-3 * rng.standard_normal(16)[:, None, None])
    f, _ = ob.run(f0, 0.0, n)
    m = ob.macros(f0)  # the conserved moments, and so f_hat^eq, stay those of f0
    q = ob.feq_moments(m["rho"][0, 0], m["ux"][0, 0], m["uy"][0, 0], m["T"][0, 0])
    d0 = ob.M @ f0[:, 0, 0] - q
    d = ob.M @ f[:, 0, 0] - q
    z = -S * dt
    R = {0: 1 + z, 1: 1 + z + z * z / 2, 2: 1 + z + z * z / 2 + z ** 3 / 6}[scheme]
    want = R ** n * d0
    assert np.all(np.abs(d[4:] - want[4:]) <= 1e-10 * np.abs(d0[4:]).max())
    assert np.abs(d[:4]).max() <= 1e-12 * np.abs(q).max()


def test_exact_riemann_solver_satisfies_jump_conditions():
    """The reference solver itself: Rankine-Hugoniot across the Sod shock and the
    isentropic relation across the rarefaction."""
    g = 1.4
    L, R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    ps, us = er.star_state(L, R, g)
    xi = np.linspace(-2, 2, 4001)
    r, u, p = er.sample(L, R, g, xi)
    idx = np.where(np.abs(np.diff(r)) > 1e-3)[0]
    k = idx[-1]  # the shock is the last jump
    s = xi[k]
    r1, u1, p1, r2, u2, p2 = r[k], u[k], p[k], r[k + 1], u[k + 1], p[k + 1]
    assert abs(r1 * (u1 - s) - r2 * (u2 - s)) < 2e-3
    assert abs(r1 * (u1 - s) ** 2 + p1 - r2 * (u2 - s) ** 2 - p2) < 4e-3
    mid = (xi > -1.0) & (xi < -0.1)
    assert np.allclose(p[mid] / r[mid] ** g, 1.0, rtol=1e-10)
    assert 0.3 < ps < 0.31 and 0.92 < us < 0.93


def test_cj_state_matches_paper_values():
    """The CJ closed form used to build the driver state reproduces the paper's printed
    CJ state and speed (Sec. IV.A)."""
    g = read_golden("cj_detonation.txt")
    D, rho, u, p, T = li.cj_state(1.0, 1.4)
    assert abs(rho - g["rho"]) < 6e-6 and abs(T - g["T"]) < 6e-6
    assert abs(u - g["u_x"]) < 6e-7 and abs(D - g["D"]) < 6e-6


@pytest.mark.slow
def test_detonation_follows_cj_theory(oracle_mod):
    """A resolved detonation (reaction zone over several cells) runs at the CJ speed, leaves
    the CJ state behind it and peaks below the ZND von Neumann pressure (Sec. IV.A)."""
    dx, dt, steps, nx = 1e-4, 2e-6, 10000, 600
    c = li.detonation(nx=nx, steps=1000, omega1=2e3, dx=dx, dt=dt)
    p = dict(c["params"])
    p.pop("nx"), p.pop("ny")
    ob = oracle_mod.Oracle(nx, 1, **p)
    fl = c["fields"]
    f = ob.init(fl["rho"], fl["ux"], fl["uy"], fl["T"])
    lam = fl["lam"]
    ts, xs, pmax = [], [], []
    for k in range(steps // 1000):
        f, lam = ob.run(f, lam, 1000)
        pr = ob.macros(f)["p"][0]
        jp = int(np.argmax(pr))
        ts.append((k + 1) * 1000 * dt)
        xs.append((jp + np.argmax(pr[jp:] < 1.5)) * dx)
        pmax.append(pr[jp])
    Dcj, rcj, ucj, pcj, Tcj = li.cj_state(1.0, 1.4)
    speed = np.polyfit(ts[4:], xs[4:], 1)[0]
    assert abs(speed / Dcj - 1) < 0.01
    m = ob.macros(f)
    j = int(xs[-1] / dx)
    seg = slice((50 + j) // 2 - 20, (50 + j) // 2 + 20)
    for k, ref in (("rho", rcj), ("ux", ucj), ("T", Tcj), ("p", pcj)):
        assert abs(m[k][0][seg].mean() / ref - 1) < 0.005, k
    assert pcj < pmax[-1] < li.von_neumann_pressure(1.0, 1.4)


def test_shear_wave_decays_at_viscous_rate(oracle_mod):
    """u_y = A sin(k x) decays at nu k^2 with nu = T/R_6 (momentum equation of Sec. III)."""
    rates = []
    for S6 in (100.0, 200.0):
        nx = 128
        S = np.full(16, 1e3)
        S[4:7] = S6
        ob = make(oracle_mod, nx, 1, S=S, dx=1.0 / nx, dt=2e-4, bc_x=0)
        x = (np.arange(nx) + 0.5) / nx
        A = 0.01
        f = ob.init(1.0, 0.0, (A * np.sin(2 * np.pi * x))[None, :], 1.0)
        f, _ = ob.run(f, 0.0, 2000)
        amp = 2 * np.mean(ob.macros(f)["uy"][0] * np.sin(2 * np.pi * x))
        rates.append(-np.log(amp / A) / 0.4)
        assert abs(rates[-1] / ((1.0 / S6) * (2 * np.pi) ** 2) - 1) < 0.04


def test_one_dimensional_symmetry_zeros(oracle_mod):
    """In a flow uniform in y the shear and y-flux non-equilibria vanish (Sec. VI):
    Delta_6, Delta_9, Delta_11, Delta_13, Delta_15 = 0."""
    c = li.detonation(nx=200, driver=40)
    p = dict(c["params"])
    p.pop("nx"), p.pop("ny")
    ob = oracle_mod.Oracle(200, 1, **p)
    fl = c["fields"]
    f = ob.init(fl["rho"], fl["ux"], fl["uy"], fl["T"])
    f, lam = ob.run(f, fl["lam"], 200)
    delta, rec = ob.tne(f)
    big = np.abs(delta).max()
    assert big > 1e-3
    for k in (5, 8, 10, 12, 14):
        assert np.abs(delta[k]).max() < 1e-12 * big


@pytest.mark.slow
def test_couette_viscous_heating_fixes_the_sign_of_A(oracle_mod):
    """Steady Couette flow between walls at T1 = 1 and T2 = 1.01, the top one moving at
    u0 = 0.3 (Sec. IV.D, non-equilibrium extrapolation walls), Pr = R_kappa/R_mu = 5:
    viscous heating bends the temperature profile upward by (Pr u0^2 / (2 c_p)) eta(1-eta)
    on top of the linear conduction profile (the Chapman-Enskog balance kappa T'' =
    -mu u'^2 of Sec. III). With the sign of A_hat taken from the Chapman-Enskog form
    Eq. (29) the fitted bump is positive and of that size (0.75x on this 20-cell channel);
    with the sign of Eq. (1) it comes out negative (-0.61x): the profile cools in the
    middle, which no heat-conducting flow does."""
    ny, dy, dt, u0, T1, T2, Pr, Rmu = 20, 1e-3, 1e-5, 0.3, 1.0, 1.01, 5.0, 2e3
    S = np.full(16, 5e4)
    S[4:7] = Rmu
    S[7:9] = Pr * Rmu
    ob = make(oracle_mod, 1, ny, S=S, dx=dy, dy=dy, dt=dt, bc_x=0, bc_y=2,
              walls=((0.0, 0.0, T1), (u0, 0.0, T2)))
    eta = ((np.arange(ny) + 0.5) / ny)[:, None]
    f = ob.init(1.0, u0 * eta, 0.0, T1 + (T2 - T1) * eta)
    f, _ = ob.run(f, np.zeros((ny, 1)), 200000)  # t = 2: steady to 1e-4 of the bump
    T = ob.macros(f)["T"][:, 0]
    e = eta[:, 0]
    coef = np.linalg.lstsq(np.stack([np.ones_like(e), e, e * (1 - e)], 1), T, rcond=None)[0]
    cp = (2 + ob.p.I + 2) / 2
    ratio = coef[2] / (Pr * u0 ** 2 / (2 * cp))
    assert 0.6 < ratio < 1.2, ratio


def test_entropy_mode_decays_at_the_thermal_diffusivity(oracle_mod):
    """A temperature ripple at uniform pressure (an entropy mode) decays at alpha k^2 with
    alpha = kappa / (rho c_p) = T / R_kappa, R_kappa = R_8 = R_9 (the energy equation of
    Sec. III; Pr = R_kappa / R_mu, Eq. (86)): independent of R_5..R_7 and halved when
    R_kappa doubles. Measured within 3 % on 128 cells (the rest is the scheme's own
    diffusion); the bound is 6 %."""
    nx, A = 128, 0.01
    x = (np.arange(nx) + 0.5) / nx
    T0 = 1 + A * np.cos(2 * np.pi * x)
    for Rmu, Rk in ((1000.0, 200.0), (200.0, 200.0), (1000.0, 400.0)):
        S = np.full(16, 2e3)
        S[4:7] = Rmu
        S[7:9] = Rk
        ob = make(oracle_mod, nx, 1, S=S, dx=1.0 / nx, dt=1e-4, bc_x=0)
        f = ob.init((1.0 / T0)[None], 0.0, 0.0, T0[None])
        lam = np.zeros((1, nx))
        amps = []
        for _ in range(4):
            f, lam = ob.run(f, lam, 2500)
            T = ob.macros(f)["T"][0]
            amps.append(2 * np.mean((T - T.mean()) * np.cos(2 * np.pi * x)))
        rate = -np.polyfit(0.25 * np.arange(1, 5), np.log(np.abs(amps)), 1)[0]
        assert abs(rate / ((2 * np.pi) ** 2 / Rk) - 1) < 0.06, (Rmu, Rk, rate)
