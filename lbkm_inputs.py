"""Seeded synthetic inputs for the MRT-LBKM combustion step.

This module is shared by the tests, the benchmark and the smoke check. It holds
only initial fields and parameters (no arithmetic of the kinetic model), so the
oracle and the CUDA path stay independent of each other. Every workload is an
analytic initial-value problem of the kind the paper runs in Sec. IV:

* ``riemann``    -- Sod-type shock tube, no reaction (Sec. IV.B).
* ``detonation`` -- 1-D detonation driven by a Chapman-Jouguet state (Sec. IV.A).
* ``reactive2d`` -- 2-D periodic reactive field of random Fourier modes.
* ``batched``    -- many 1-D detonations of uneven length and differing S, Q.
* ``adjoint``    -- 1-D detonation whose target is a run with perturbed S, Q.
* ``lax``, ``sjogreen`` -- the other two shock tubes of Sec. IV.B.
* ``couette``    -- Couette flow between walls (Sec. IV.D).
* ``shock_reflection`` -- regular reflection of an oblique shock on a wall (Sec. IV.C).
* ``d2v24_detonation``, ``d2v24_reactive2d`` -- the same kinds of problem for the
  paper's own 24-velocity model D2V24 (Sec. II, Eqs. (25)-(27)), with the paper's
  velocity parameters (v_a, v_b, v_c; eta_a, eta_b, eta_c).

Default velocity set: a 16-velocity model of four orbits (axis, diagonal, axis,
diagonal) with speeds (2.7, 2.2, 1.2, 1.0) and eta (5, 0, 3, 0). The paper's
24-velocity set cut to its first two rings gives a singular 16x16 M (rank 14),
so the 16-velocity model uses four orbits with their own speeds instead.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 14116697

DEFAULT_ORBITS = dict(orbit_kind=(0, 1, 0, 1), orbit_speed=(2.7, 2.2, 1.2, 1.0),
                      orbit_eta=(5.0, 0.0, 3.0, 0.0))


# (v_a, v_b, v_c), (eta_a, eta_b, eta_c) of the paper's D2V24 runs
D2V24_DETONATION_V = ((2.7, 2.2, 1.2), (5.0, 3.0, 1.1))    # steady detonation, Sec. IV.A
D2V24_TNE_V = ((2.7, 2.2, 1.2), (1.5, 0.5, 5.0))           # TNE study, Sec. VI (R_i = 100)
D2V24_TNE_V2 = ((2.7, 2.6, 1.9), (5.0, 0.0, 1.7))          # Sec. VI, R_i = 1e3 and 1e4


def d2v24_orbits(v, eta):
    """Six-orbit table (axis and diagonal at each of v_a, v_b, v_c) of a D2V24 set."""
    return dict(orbit_kind=(0, 1, 0, 1, 0, 1),
                orbit_speed=(v[0], v[0], v[1], v[1], v[2], v[2]),
                orbit_eta=(eta[0], eta[0], eta[1], eta[1], eta[2], eta[2]))


def cj_state(Q: float, gamma: float, rho0: float = 1.0, p0: float = 1.0):
    """Chapman-Jouguet detonation into a gas at rest (rho0, p0) with heat release Q
    per unit mass (ideal gas, specific internal energy p/((gamma-1) rho)).

    Returns (D_cj, rho, u, p, T) of the burnt state, T = p/rho. Closed form of the
    Rayleigh line tangent to the equilibrium Hugoniot (CJ theory cited in Sec. IV.A).
    """
    c0sq = gamma * p0 / rho0
    q = (gamma * gamma - 1.0) * Q / c0sq
    M2 = 1.0 + q + math.sqrt((1.0 + q) ** 2 - 1.0)
    Dcj = math.sqrt(M2 * c0sq)
    p = p0 * (1.0 + gamma * M2) / (1.0 + gamma)
    rho = rho0 * (gamma + 1.0) * M2 / (1.0 + gamma * M2)
    u = Dcj * (1.0 - rho0 / rho)
    return Dcj, rho, u, p, p / rho


def von_neumann_pressure(Q: float, gamma: float, rho0: float = 1.0, p0: float = 1.0):
    """Pressure behind a non-reacting shock moving at the CJ speed (ZND spike)."""
    c0sq = gamma * p0 / rho0
    Dcj = cj_state(Q, gamma, rho0, p0)[0]
    M2 = Dcj * Dcj / c0sq
    return p0 * (2.0 * gamma * M2 - (gamma - 1.0)) / (gamma + 1.0)


def _base(**kw):
    d = dict(DEFAULT_ORBITS)
    d.update(gamma=1.4, Q=0.0, omega1=0.0, omega2=0.0, T_ig=1.1, bc_x=1, bc_y=0, ny=1)
    d.update(kw)
    return d


def riemann(nx=400, steps=1000, run="A", interface=None):
    """Sod shock tube on nx cells: left rho=1, p=1; right rho=0.125, p=0.1; u=0.
    Run A: all S = 1e5 (single-relaxation limit). Run B: S uniform in [0.8e5, 1.2e5]."""
    rng = np.random.default_rng(SEED_BASE + 1)
    S = np.full(16, 1e5) if run == "A" else rng.uniform(0.8e5, 1.2e5, 16)
    iface = nx // 2 if interface is None else interface
    rho = np.where(np.arange(nx) < iface, 1.0, 0.125)[None, :]
    T = np.where(np.arange(nx) < iface, 1.0, 0.8)[None, :]
    zero = np.zeros((1, nx))
    return dict(params=_base(nx=nx, S=S, dx=1e-3, dt=1e-5), steps=steps,
                fields=dict(rho=rho, ux=zero, uy=zero.copy(), T=T, lam=zero.copy()),
                name="riemann%s_nx%d" % (run, nx))


def _shock_tube(nx, steps, dx, dt, gamma, S, left, right, name):
    """Two constant states (rho, T, u_x) meeting at the middle of the grid."""
    x = np.arange(nx)
    L = x < nx // 2
    rho = np.where(L, left[0], right[0])[None, :]
    T = np.where(L, left[1], right[1])[None, :]
    ux = np.where(L, left[2], right[2])[None, :]
    zero = np.zeros((1, nx))
    return dict(params=_base(nx=nx, S=np.asarray(S, float), dx=dx, dt=dt, gamma=gamma),
                steps=steps, fields=dict(rho=rho, ux=ux, uy=zero, T=T, lam=zero.copy()),
                name=name, left=left, right=right)


def lax(nx=2000, steps=15000):
    """Lax shock tube (Sec. IV.B): (rho, T, u_x) = (0.445, 7.928, 0.698) | (0.5, 1.142, 0)
    on [-1, 1], dx = 1e-3, dt = 1e-5, t = 0.15, I = 1 (gamma = 5/3), R_5..R_7 = 2e4,
    R_8 = R_9 = 8e4, other R = 1e5. The left gas is eight times hotter than in the other
    tests, so the orbit speeds are widened by 1.5 (the paper widens its own velocity set
    for this test too); with the default speeds the run amplifies a 1e-15 perturbation
    to 3e-4 by t = 0.15, with the widened ones to 5e-9."""
    S = np.full(16, 1e5)
    S[4:7] = 2e4
    S[7:9] = 8e4
    c = _shock_tube(nx, steps, 1e-3, 1e-5, 5.0 / 3.0, S, (0.445, 7.928, 0.698),
                    (0.5, 1.142, 0.0), "lax_nx%d" % nx)
    c["params"]["orbit_speed"] = [1.5 * v for v in c["params"]["orbit_speed"]]
    return c


def sjogreen(nx=500, steps=1500):
    """Sjogreen's problem (Sec. IV.B): (rho, T, u_x) = (1, 0.5, -1.2) | (1, 0.5, 1.2) on
    [-0.5, 0.5], dx = 2e-3, dt = 2e-5, t = 0.03, I = 4 (gamma = 4/3), R_8 = R_9 = 2e4,
    other R = 5e4."""
    S = np.full(16, 5e4)
    S[7:9] = 2e4
    return _shock_tube(nx, steps, 2e-3, 2e-5, 4.0 / 3.0, S, (1.0, 0.5, -1.2),
                       (1.0, 0.5, 1.2), "sjogreen_nx%d" % nx)


def couette(ny=200, steps=50000, u0=0.1, nx=1):
    """Couette flow (Sec. IV.D): walls at y = 0 (at rest) and y = H = ny dy (moving at
    u0), non-equilibrium extrapolation at both, periodic x; rho = 1, T = 1, u = 0 at
    t = 0; dy = 1e-3, dt = 1e-5, I = 2 (gamma = 1.5), R_5..R_7 = 2e3, R_8 = R_9 = 1e4,
    other R = 5e4. 50000 steps reach t = 0.5 (nu t / H^2 = 0.00625)."""
    S = np.full(16, 5e4)
    S[4:7] = 2e3
    S[7:9] = 1e4
    p = _base(nx=nx, ny=ny, S=S, dx=1e-3, dt=1e-5, gamma=1.5, bc_x=0, bc_y=2)
    p["walls"] = ((0.0, 0.0, 1.0), (u0, 0.0, 1.0))
    one, zero = np.ones((ny, nx)), np.zeros((ny, nx))
    return dict(params=p, steps=steps, u0=u0,
                fields=dict(rho=one, ux=zero, uy=zero.copy(), T=one.copy(), lam=zero.copy()),
                name="couette_ny%d" % ny)


def shock_reflection(nx=300, ny=100, steps=100000):
    """Regular shock reflection (Sec. IV.C): a 0.3 x 0.1 box of 300 x 100 cells, dx = dy
    = 1e-3, dt = 5e-6 (100000 steps reach t = 0.5), I = 2 (gamma = 1.5); R_5..R_7 =
    1.8e5, R_8 = R_9 = 2e5, other R = 1e5. Dirichlet inflow (rho, T, u_x, u_y) =
    (1, 0.5, 2, 0) at x = 0 and the post-shock state (1.25, 0.56, 1.9, -0.173205) on the
    top, supersonic outflow (zero gradient) at x = 0.3, a specular wall at y = 0. The
    box starts filled with the inflow state. Orbit speeds (3.0, 2.9, 1.0, 1.0) and eta
    (2.5, 0, 1.5, 0): with the default table the uniform Mach-2.3 inflow itself grows
    rounding noise to NaN within 3000 steps; this table keeps it to 3e-14 for 20000."""
    S = np.full(16, 1e5)
    S[4:7] = 1.8e5
    S[7:9] = 2e5
    p = _base(nx=nx, ny=ny, S=S, dx=1e-3, dt=5e-6, gamma=1.5, bc_x=5, bc_y=5)
    p["orbit_speed"] = [3.0, 2.9, 1.0, 1.0]
    p["orbit_eta"] = [2.5, 0.0, 1.5, 0.0]
    # (code, rho, ux, uy, T, lambda) of the sides x = 0, x = nx, y = 0, y = ny
    p["sides"] = ((3, 1.0, 2.0, 0.0, 0.5, 0.0), (1, 1.0, 0.0, 0.0, 1.0, 0.0),
                  (4, 1.0, 0.0, 0.0, 1.0, 0.0), (3, 1.25, 1.9, -0.173205, 0.56, 0.0))
    one, zero = np.ones((ny, nx)), np.zeros((ny, nx))
    return dict(params=p, steps=steps,
                fields=dict(rho=one, ux=2.0 * one, uy=zero, T=0.5 * one, lam=zero.copy()),
                name="shock_reflection_%dx%d" % (nx, ny))


def detonation(nx=16384, steps=20000, driver=50, Q=1.0, S=None, dx=1e-4, dt=2e-6,
               omega1=2e4, gamma=1.4, ripple=0.0):
    """1-D detonation: CJ burnt state (lambda=1) in the first `driver` cells, unburnt
    premix rho=1, T=1, u=0, lambda=0 ahead. S_5..S_7 = 1e4, the others 1e5 (Sec. IV.A).

    ripple > 0 multiplies rho and T by 1 + ripple * r(x), with independent r for each, a
    seeded sum of four long sine modes (|r| <= 1), so that no two neighbouring cells hold
    equal or nearly equal states: every
    minmod branch is then decided by differences far above rounding, which makes the
    gradient of the discrete map a well-posed comparison between implementations."""
    if S is None:
        S = np.full(16, 1e5)
        S[4:7] = 1e4
    _, rcj, ucj, _, Tcj = cj_state(Q, gamma)
    burnt = np.arange(nx) < driver
    f = dict(rho=np.where(burnt, rcj, 1.0)[None, :], ux=np.where(burnt, ucj, 0.0)[None, :],
             uy=np.zeros((1, nx)), T=np.where(burnt, Tcj, 1.0)[None, :],
             lam=np.where(burnt, 1.0, 0.0)[None, :])
    if ripple > 0.0:
        rng = np.random.default_rng(SEED_BASE + 6)
        x = np.arange(nx) / nx

        def r():
            amp, ph = rng.uniform(0.5, 1.0, 4), rng.uniform(0, 2 * np.pi, 4)
            s = sum(a * np.sin(2 * np.pi * (k + 1) * x + p)
                    for k, (a, p) in enumerate(zip(amp, ph)))
            return s / np.abs(s).max()
        # independent ripples: with T tied to rho some f_i would be flat to first order
        f["rho"] = f["rho"] * (1.0 + ripple * r())
        f["T"] = f["T"] * (1.0 + ripple * r())
    return dict(params=_base(nx=nx, S=np.asarray(S, float), Q=Q, omega1=omega1, T_ig=1.1,
                             dx=dx, dt=dt, gamma=gamma),
                steps=steps, fields=f, name="detonation_nx%d" % nx)


def d2v24_detonation(nx=5000, steps=78000, omega1=1e3, dx=2e-4, dt=5e-6, S=None,
                     v=D2V24_DETONATION_V, x_driver=0.2, ripple=0.0):
    """The steady-detonation run of Sec. IV.A with D2V24: x in [0, nx dx), the paper's
    printed burnt state (rho, T, u_x, lambda) = (1.38837, 1.57856, 0.577350, 1) for
    x <= x_driver and (1, 1, 0, 0) beyond, gamma = 1.4 (I = 3), Q = 1, T_ig = 1.1,
    R_5..R_7 = 1e4 and the others 1e5, dx = 2e-4, dt = 5e-6 (t = 0.39 after 78000
    steps). The paper leaves the rate constant unstated: omega1 = 1e3 here. With 2e4 at
    this dx the premix ahead of the shock, heated past T_ig by the fastest particles,
    burns first and the burn front outruns the shock (about 2.47 against 2.06), which
    the paper's printed speed rules out.
    Returns params for the D2V24 oracle (six orbits) and for lbkm24 (v, eta, S[24])."""
    if S is None:
        S = np.full(24, 1e5)
        S[4:7] = 1e4
    burnt = (np.arange(nx) * dx) <= x_driver + 1e-12
    f = dict(rho=np.where(burnt, 1.38837, 1.0)[None, :],
             ux=np.where(burnt, 0.577350, 0.0)[None, :], uy=np.zeros((1, nx)),
             T=np.where(burnt, 1.57856, 1.0)[None, :], lam=np.where(burnt, 1.0, 0.0)[None, :])
    if ripple > 0.0:
        rng = np.random.default_rng(SEED_BASE + 7)
        x = np.arange(nx) / nx
        for k in ("rho", "T"):
            amp, ph = rng.uniform(0.5, 1.0, 4), rng.uniform(0, 2 * np.pi, 4)
            r = sum(a * np.sin(2 * np.pi * (j + 1) * x + p) for j, (a, p) in enumerate(zip(amp, ph)))
            f[k] = f[k] * (1.0 + ripple * r / np.abs(r).max())
    common = dict(nx=nx, ny=1, gamma=1.4, Q=1.0, omega1=omega1, omega2=0.0, T_ig=1.1, dx=dx,
                  dy=dx, dt=dt, bc_x=1, bc_y=0)
    oracle_params = dict(common, S=np.asarray(S, float), **d2v24_orbits(*v))
    lib_params = dict(common, S=np.asarray(S, float), v=v[0], eta=v[1])
    return dict(params=oracle_params, lib_params=lib_params, steps=steps, fields=f,
                name="d2v24_detonation_nx%d" % nx)


# The paper leaves the rate constant of its Sec. VI detonations unstated. With omega1 = 13
# its case (i) reaches, at t = 0.35, a pressure peak of 2.405 at x = 0.784 (printed: 2.3985
# at 0.8345); from omega1 ~ 18 upwards a weak reaction front, lit inside the thick shock of
# the R_i = 1e2 gas, outruns the detonation and the peak stays at the initial interface.
D2V24_SEC6_OMEGA1 = 13.0


def d2v24_tne_study(case=1, omega1=D2V24_SEC6_OMEGA1):
    """The detonations of Sec. VI with D2V24, run to t = 0.35 from the initial state of
    Sec. IV.A on x in [0, 1): case 1, R_i = 1e2 with v = (2.7, 2.2, 1.2), eta = (1.5,
    0.5, 5.0), dx = 1e-3, dt = 1e-5; case 2, R_i = 1e3 with v = (2.7, 2.6, 1.9), eta =
    (5.0, 0.0, 1.7), dx = 2e-4, dt = 2e-6; case 3, R_i = 1e4 with the case-2 set, dx =
    4e-5, dt = 4e-6. All R_i equal (the section's collision parameters); I = 3, Q = 1,
    T_ig = 1.1 as in Sec. IV.A."""
    R, v, dx, dt = {1: (1e2, D2V24_TNE_V, 1e-3, 1e-5),
                    2: (1e3, D2V24_TNE_V2, 2e-4, 2e-6),
                    3: (1e4, D2V24_TNE_V2, 4e-5, 4e-6)}[case]
    nx, steps = int(round(1.0 / dx)), int(round(0.35 / dt))
    c = d2v24_detonation(nx=nx, steps=steps, omega1=omega1, dx=dx, dt=dt, S=np.full(24, R), v=v)
    c["name"] = "d2v24_sec6_case%d" % case
    return c


def d2v24_shock_tube(which, steps=None):
    """The three shock tubes of Sec. IV.B with the paper's own D2V24 sets:
    Sod: (1, 1, 0) | (0.125, 0.8, 0) on [0, 1], 1000 cells, dt = 1e-5, t = 0.2, I = 3,
    (v; eta) = (2.5, 2.2, 1.2; 6.5, 3, 0), R_5..R_7 = 1.2e4, others 1e5;
    Lax: (0.445, 7.928, 0.698) | (0.5, 1.142, 0) on [-1, 1], 2000 cells, dt = 1e-5,
    t = 0.15, I = 1, (4.7, 3.3, 1; 6, 2.5, 0.9), R_5..R_7 = 2e4, R_8, R_9 = 8e4, others 1e5;
    Sjogreen: (1, 0.5, -1.2) | (1, 0.5, 1.2) on [-0.5, 0.5], 500 cells, dt = 2e-5,
    t = 0.03, I = 4, (0.4, 1.0, 1.8; 0.3, 1.9, 1.5), R_8, R_9 = 2e4, others 5e4.
    States are (rho, T, u_x); steps defaults to the paper's end time."""
    S = np.full(24, 1e5)
    if which == "sod":
        S[4:7] = 1.2e4
        nx, dx, dt, t, gamma, v = 1000, 1e-3, 1e-5, 0.2, 1.4, ((2.5, 2.2, 1.2), (6.5, 3.0, 0.0))
        left, right = (1.0, 1.0, 0.0), (0.125, 0.8, 0.0)
    elif which == "lax":
        S[4:7] = 2e4
        S[7:9] = 8e4
        nx, dx, dt, t, gamma, v = 2000, 1e-3, 1e-5, 0.15, 5.0 / 3.0, ((4.7, 3.3, 1.0), (6.0, 2.5, 0.9))
        left, right = (0.445, 7.928, 0.698), (0.5, 1.142, 0.0)
    else:
        S[:] = 5e4
        S[7:9] = 2e4
        nx, dx, dt, t, gamma, v = 500, 2e-3, 2e-5, 0.03, 4.0 / 3.0, ((0.4, 1.0, 1.8), (0.3, 1.9, 1.5))
        left, right = (1.0, 0.5, -1.2), (1.0, 0.5, 1.2)
    x = np.arange(nx)
    L = x < nx // 2
    fields = dict(rho=np.where(L, left[0], right[0])[None, :],
                  T=np.where(L, left[1], right[1])[None, :],
                  ux=np.where(L, left[2], right[2])[None, :], uy=np.zeros((1, nx)),
                  lam=np.zeros((1, nx)))
    common = dict(nx=nx, ny=1, gamma=gamma, Q=0.0, omega1=0.0, omega2=0.0, T_ig=1.1, dx=dx,
                  dy=dx, dt=dt, bc_x=1, bc_y=0)
    n = int(round(t / dt)) if steps is None else steps
    return dict(params=dict(common, S=S, **d2v24_orbits(*v)),
                lib_params=dict(common, S=S, v=v[0], eta=v[1]), steps=n, fields=fields,
                left=left, right=right, name="d2v24_%s_nx%d" % (which, nx))


def d2v24_shock_reflection(steps=100000, nx=300, ny=100):
    """The regular shock reflection of Sec. IV.C with the paper's own D2V24 set:
    (v_a, v_b, v_c; eta_a, eta_b, eta_c) = (1.0, 2.7, 2.9; 1.0, 2.9, 0.96), I = 2
    (gamma = 1.5), dt = 5e-6, dx = dy = 1e-3 on a 0.3 x 0.1 box (100000 steps reach
    t = 0.5), R_5..R_7 = 1.8e5, R_8 = R_9 = 2e5, others 1e5; Dirichlet inflow (rho, T, u_x,
    u_y) = (1, 0.5, 2, 0) at x = 0 and the post-shock state (1.25, 0.56, 1.9, -0.173205)
    on the top, zero-gradient outflow at x = 0.3, a specular wall at y = 0; the box starts
    filled with the inflow state."""
    S = np.full(24, 1e5)
    S[4:7] = 1.8e5
    S[7:9] = 2e5
    v = ((1.0, 2.7, 2.9), (1.0, 2.9, 0.96))
    sides = ((3, 1.0, 2.0, 0.0, 0.5, 0.0), (1, 1.0, 0.0, 0.0, 1.0, 0.0),
             (4, 1.0, 0.0, 0.0, 1.0, 0.0), (3, 1.25, 1.9, -0.173205, 0.56, 0.0))
    common = dict(nx=nx, ny=ny, gamma=1.5, Q=0.0, omega1=0.0, omega2=0.0, T_ig=1.1, dx=1e-3,
                  dy=1e-3, dt=5e-6, bc_x=5, bc_y=5, sides=sides)
    one, zero = np.ones((ny, nx)), np.zeros((ny, nx))
    return dict(params=dict(common, S=S, **d2v24_orbits(*v)),
                lib_params=dict(common, S=S, v=v[0], eta=v[1]), steps=steps,
                fields=dict(rho=one, ux=2.0 * one, uy=zero, T=0.5 * one, lam=zero.copy()),
                name="d2v24_shock_reflection_%dx%d" % (nx, ny))


def d2v24_couette(ny=200, steps=100000, u0=0.1):
    """Couette flow of Sec. IV.D with the paper's own D2V24 set: 1 x 200 cells, dy = 1e-3
    (H = 0.2), dt = 1e-5, I = 2 (gamma = 1.5), (v; eta) = (0.8, 1.2, 1.3; 1.0, 2.7, 0.8),
    R_5..R_7 = 2e3, R_8 = R_9 = 1e4, others 5e4; walls by non-equilibrium extrapolation,
    the lower at rest, the upper moving at u0, both at T = 1; periodic in x; the fluid
    starts at rest with rho = 1, T = 1. With this set the moving wall's non-equilibrium
    extrapolation grows an instability next to it within a few hundred steps (u_x there
    turns negative, then non-finite; a wall at rest and a periodic shear stay bounded),
    in the oracle as on the GPU."""
    S = np.full(24, 5e4)
    S[4:7] = 2e3
    S[7:9] = 1e4
    v = ((0.8, 1.2, 1.3), (1.0, 2.7, 0.8))
    sides = ((1, 1.0, 0.0, 0.0, 1.0, 0.0), (1, 1.0, 0.0, 0.0, 1.0, 0.0),
             (2, 1.0, 0.0, 0.0, 1.0, 0.0), (2, 1.0, u0, 0.0, 1.0, 0.0))
    common = dict(nx=1, ny=ny, gamma=1.5, Q=0.0, omega1=0.0, omega2=0.0, T_ig=1.1, dx=1e-3,
                  dy=1e-3, dt=1e-5, bc_x=0, bc_y=5, sides=sides)
    one, zero = np.ones((ny, 1)), np.zeros((ny, 1))
    oracle_params = dict(common, S=S, walls=((0.0, 0.0, 1.0), (u0, 0.0, 1.0)),
                         **d2v24_orbits(*v))
    return dict(params=oracle_params, lib_params=dict(common, S=S, v=v[0], eta=v[1]),
                steps=steps, u0=u0,
                fields=dict(rho=one, ux=zero, uy=zero.copy(), T=one.copy(), lam=zero.copy()),
                name="d2v24_couette_1x%d" % ny)


def d2v24_reactive2d(n=64, steps=20, T_ig=1.0, seed_offset=8, v=D2V24_DETONATION_V):
    """2-D periodic reactive field of random Fourier modes (the recipe of reactive2d)
    for D2V24: S_1..S_24 ~ U[1e4, 1e5], Q = 1, k = 2e4, dx = dy = 1e-3, dt = 5e-6."""
    base = reactive2d(n=n, steps=steps, T_ig=T_ig, seed_offset=seed_offset)
    rng = np.random.default_rng(SEED_BASE + seed_offset + 100)
    S = rng.uniform(1e4, 1e5, 24)
    common = dict(nx=n, ny=n, gamma=1.4, Q=1.0, omega1=2e4, omega2=0.0, T_ig=T_ig, dx=1e-3,
                  dy=1e-3, dt=5e-6, bc_x=0, bc_y=0)
    return dict(params=dict(common, S=S, **d2v24_orbits(*v)),
                lib_params=dict(common, S=S, v=v[0], eta=v[1]), steps=steps,
                fields=base["fields"], name="d2v24_reactive2d_%dx%d" % (n, n))


def _modes(rng, nmodes, kmax):
    ks = []
    while len(ks) < nmodes:
        k = rng.integers(-kmax, kmax + 1, size=2)
        if 1 <= math.hypot(*k) <= kmax:
            ks.append(k)
    return np.array(ks), rng.uniform(0, 1, nmodes), rng.uniform(0, 2 * np.pi, nmodes)


def _mode_sum(ks, amp, ph, nx, ny, deriv=None):
    """sum_m a_m cos(2 pi (kx x/nx + ky y/ny) + theta_m) on the grid, or its x / y
    derivative in grid units. cos(A + B) = cos A cos B - sin A sin B makes the sum
    two rank-32 products of per-axis tables."""
    xs, ys = np.arange(nx) / nx, np.arange(ny) / ny
    ax = 2 * np.pi * np.outer(ks[:, 0], xs) + ph[:, None]   # [m, nx]
    ay = 2 * np.pi * np.outer(ks[:, 1], ys)                  # [m, ny]
    cx, sx, cy, sy = np.cos(ax), np.sin(ax), np.cos(ay), np.sin(ay)
    if deriv is None:
        w = amp
        return (cy.T * w) @ cx - (sy.T * w) @ sx
    w = amp * (ks[:, 0] if deriv == "x" else ks[:, 1])
    # d/dk of cos(A + B) = -sin(A + B) = -(sin B cos A + cos B sin A)
    return -((sy.T * w) @ cx + (cy.T * w) @ sx)


def reactive2d(n=4096, steps=500, T_ig=1.0, seed_offset=3, ny=None):
    """2-D periodic reactive field on n x n cells (n x ny with ny): rho, T = 1 + 0.05
    phi/max|phi| with phi a sum of 32 random Fourier modes (1 <= |k| <= 16), solenoidal u
    of peak 0.1 from a second mode set, lambda ~ U[0, 0.2], S ~ U[1e4, 1e5], Q = 1, k = 2e4.
    T_ig defaults to 1.0: with T <= 1.05 the paper's 1.1 would leave the field inert."""
    rng = np.random.default_rng(SEED_BASE + seed_offset)
    nx, ny = n, (n if ny is None else ny)
    kmax = min(16, min(nx, ny) // 4)
    fields = {}
    for name in ("rho", "T"):
        phi = _mode_sum(*_modes(rng, 32, kmax), nx, ny)
        fields[name] = 1.0 + 0.05 * phi / np.abs(phi).max()
    ks, amp, ph = _modes(rng, 32, kmax)
    ux = _mode_sum(ks, amp, ph, nx, ny, deriv="y")
    uy = -_mode_sum(ks, amp, ph, nx, ny, deriv="x")
    if nx != ny:  # u = (d/dy, -d/dx) of the stream function, each axis in its own units
        ux, uy = ux / ny, uy / nx
    umax = np.sqrt(ux * ux + uy * uy).max()
    fields["ux"], fields["uy"] = 0.1 * ux / umax, 0.1 * uy / umax
    fields["lam"] = rng.uniform(0.0, 0.2, (ny, nx))
    S = rng.uniform(1e4, 1e5, 16)
    return dict(params=_base(nx=nx, ny=ny, S=S, Q=1.0, omega1=2e4, T_ig=T_ig, dx=1e-3,
                             dt=5e-6, bc_x=0, bc_y=0),
                steps=steps, fields=fields, name="reactive2d_%dx%d" % (nx, ny))


def batched(n_instances=512, steps=5000, nx_min=1024, nx_max=65536, driver=50):
    """Many 1-D detonations: nx log-uniform in [nx_min, nx_max] (multiple of 4), Q ~
    U[0.5, 2] with the CJ driver state of each instance's own Q, dx = 1e-4, dt = 1e-6.

    Rates: the detonation structure of Sec. IV.A (S_5..S_7 = a, every other S_k = 10 a)
    with a log-uniform in [1e4, 1e5] per instance, so the S_k span [1e4, 1e6]. Drawing
    the sixteen S_k independently in [1e4, 1e6] instead gives instances that blow up
    within a few hundred steps in the FP64 oracle itself (21 of 512 by step 400: heat-flux
    rates S_8, S_9 below the viscous ones, or far above them)."""
    rng = np.random.default_rng(SEED_BASE + 4)
    nxs = np.exp(rng.uniform(np.log(nx_min), np.log(nx_max), n_instances))
    nxs = (np.round(nxs / 4) * 4).astype(np.int64)
    a = np.exp(rng.uniform(np.log(1e4), np.log(1e5), n_instances))
    S = 10.0 * a[:, None] * np.ones((1, 16))
    S[:, 4:7] = a[:, None]
    Q = rng.uniform(0.5, 2.0, n_instances)
    insts = []
    for i in range(n_instances):
        d = detonation(nx=int(nxs[i]), steps=steps, driver=driver, Q=float(Q[i]), S=S[i],
                       dx=1e-4, dt=1e-6)
        insts.append(d)
    return dict(instances=insts, steps=steps, nx=nxs, S=S, Q=Q,
                name="batched_%d" % n_instances)


def adjoint(nx=8192, steps=4000):
    """Detonation of nx cells (structure and parameters of ``detonation``, with a 1e-3
    ripple) and a target run with S_k (1 + 0.05 xi_k), Q * 1.05, xi ~ N(0, 1)."""
    rng = np.random.default_rng(SEED_BASE + 5)
    base = detonation(nx=nx, steps=steps, ripple=1e-3)
    xi = rng.standard_normal(16)
    S_t = base["params"]["S"] * (1.0 + 0.05 * xi)
    target = detonation(nx=nx, steps=steps, Q=1.05, S=S_t, ripple=1e-3)
    return dict(base=base, target=target, w_tne=1.0, checkpoint_every=64,
                name="adjoint_nx%d" % nx)
