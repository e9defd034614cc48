"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Same seeded inputs on both sides; element-wise comparison by relative L2 per
field: <= 1e-12 for the FP64 form, <= 2e-5 for the FP32 forms. Grids span
several tiles and a ragged tail (tiles are 32 x 8 cells in 2-D, 64 in 1-D).
"""
import numpy as np
import pytest

import exact_riemann as er
import lbkm_inputs as li
from oracle.oracle import unpack_tne as oracle_unpack
from gpu_common import TOL, make_oracle, rel_l2, solver, state_bytes
from paper_1411_6697_gb300 import lbkm

pytestmark = pytest.mark.gpu

PRECS = [(lbkm.F64, 0), (lbkm.F32, 0), (lbkm.F32, 1)]
PID = ["f64", "f32", "f32-df"]


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available(), "the -m gpu tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()


def mixed_2d(nx, ny, bc=(0, 0), seed=0, reactive=True):
    """A 2-D non-uniform state with shear, compression, heat release and unequal R_k."""
    rng = np.random.default_rng(seed)
    x = np.arange(nx)[None, :] / nx
    y = np.arange(ny)[:, None] / ny
    fields = dict(
        rho=1 + 0.1 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) + 0 * x,
        ux=0.2 * np.cos(2 * np.pi * y) + 0.05 * np.sin(4 * np.pi * x),
        uy=-0.15 * np.sin(2 * np.pi * x) + 0.05 * np.cos(2 * np.pi * y),
        T=1.1 + 0.15 * np.cos(2 * np.pi * (x + y)) + 0 * x,
        lam=rng.uniform(0, 0.6, (ny, nx)))
    params = dict(li.DEFAULT_ORBITS, nx=nx, ny=ny, gamma=1.4, S=rng.uniform(5e3, 1e5, 16),
                  Q=1.0 if reactive else 0.0, omega1=2e3, omega2=300.0, T_ig=1.1, dx=1e-3,
                  dt=1e-5, bc_x=bc[0], bc_y=bc[1])
    return params, fields


def start(params, fields, prec, rec, noise_seed=None, **kw):
    """Solver and oracle at the same start state; with noise_seed the state is a
    perturbed (non-equilibrium) f, loaded through lbkm_set_state."""
    ob = make_oracle(params)
    f = ob.init(fields["rho"], fields["ux"], fields["uy"], fields["T"])
    lam = np.broadcast_to(fields["lam"], f.shape[1:]).copy()
    s = solver(params, prec, rec, **kw)
    if noise_seed is None:
        s.init_fields(fields["rho"], fields["ux"], fields["uy"], fields["T"], fields["lam"])
        if prec == lbkm.F32:
            planes = s.f_planes()  # oracle starts from the same FP32-rounded state
            f, lam = planes[:16].copy(), planes[16].copy()
    else:
        rng = np.random.default_rng(noise_seed)
        f = f * (1 + 2e-3 * rng.standard_normal(f.shape))
        if prec == lbkm.F32:
            f = f.astype(np.float32).astype(np.float64)
            lam = lam.astype(np.float32).astype(np.float64)
        s.set_state(state_bytes(np.concatenate([f, lam[None]]), prec))
    return s, ob, f, lam


# ------------------------------------------------------------------ init, macros
@pytest.mark.parametrize("prec", [lbkm.F64, lbkm.F32], ids=["f64", "f32"])
def test_init_is_discrete_equilibrium(prec):
    params, fields = mixed_2d(37, 11)
    s = solver(params, prec)
    s.init_fields(fields["rho"], fields["ux"], fields["uy"], fields["T"], fields["lam"])
    ob = make_oracle(params)
    f = ob.init(fields["rho"], fields["ux"], fields["uy"], fields["T"])
    got = s.f_planes()
    tol = 1e-13 if prec == lbkm.F64 else 1e-7
    for i in range(16):
        assert rel_l2(got[i], f[i]) < tol, i
    m = s.macros()
    for k in ("rho", "ux", "uy", "T"):
        assert rel_l2(m[k], np.broadcast_to(fields[k], m[k].shape)) < (
            1e-13 if prec == lbkm.F64 else 1e-6), k
    assert np.array_equal(m["p"], m["rho"] * m["T"])


# ------------------------------------------------------------------ fused step, 2-D
@pytest.mark.parametrize("prec,rec", PRECS, ids=PID)
@pytest.mark.parametrize("nx,ny,bc", [(70, 37, (0, 0)), (45, 19, (1, 1)), (33, 9, (1, 0)),
                                      (300, 77, (0, 0)), (262, 40, (1, 1)), (130, 3, (0, 1))])
def test_step_2d_nonequilibrium_parity(prec, rec, nx, ny, bc):
    params, fields = mixed_2d(nx, ny, bc=bc, seed=nx)
    s, ob, f, lam = start(params, fields, prec, rec, noise_seed=ny)
    steps = 25
    s.step(steps)
    f_ref, lam_ref = ob.run(f, lam, steps)
    got = s.f_planes()
    for i in range(16):
        assert rel_l2(got[i], f_ref[i]) <= TOL[prec], ("f", i + 1, rel_l2(got[i], f_ref[i]))
    assert rel_l2(got[16], lam_ref) <= TOL[prec]
    m, mr = s.macros(), ob.macros(f_ref)
    for k in ("rho", "ux", "uy", "T", "p"):
        assert rel_l2(m[k], mr[k]) <= TOL[prec], (k, rel_l2(m[k], mr[k]))
    assert lam_ref.max() > lam.max() - 1e-12  # the reaction ran


# ------------------------------------------------------------------ SSP-RK2 / RK3 steps
@pytest.mark.parametrize("scheme", [1, 2], ids=["rk2", "rk3"])
@pytest.mark.parametrize("prec,rec", PRECS, ids=PID)
@pytest.mark.parametrize("nx,ny,bc", [(70, 37, (0, 0)), (262, 40, (1, 1)), (33, 9, (1, 0)),
                                      (300, 1, (1, 0))])
def test_rk_steps_parity(prec, rec, nx, ny, bc, scheme):
    """The two- and three-stage SSP Runge-Kutta schemes (fused Euler launches, the later
    ones weighted with u^n): 40 steps (one graph-captured chunk of 32 and 8 direct steps),
    every plane against the oracle's scheme, the step count and the per-step TNE of u^n."""
    params, fields = mixed_2d(nx, ny, bc=bc, seed=nx + 3)
    params["time_scheme"] = scheme
    s, ob, f, lam = start(params, fields, prec, rec, noise_seed=ny + 3, tne_every=1,
                          tne_capacity=64)
    steps = 40
    s.step(steps)
    f_ref, lam_ref, tne_ref = ob.run(f, lam, steps, tne=True)
    got = s.f_planes()
    for i in range(16):
        assert rel_l2(got[i], f_ref[i]) <= TOL[prec], ("f", i + 1, rel_l2(got[i], f_ref[i]))
    assert rel_l2(got[16], lam_ref) <= TOL[prec]
    assert s.steps_taken == steps
    hist = s.tne_history(max_records=steps)
    assert len(hist) == steps
    from oracle.oracle import unpack_tne
    for n in (0, steps // 2, steps - 1):
        ref = unpack_tne(tne_ref[n])
        scale = np.abs(ref["abs_sum"]).max()
        tol = 1e-10 if prec == lbkm.F64 else 1e-3
        assert np.abs(hist[n]["abs_sum"] - ref["abs_sum"]).max() <= tol * scale, n
        assert hist[n]["step"] == n


# ------------------------------------------------------------------ walls (Sec. IV.D)
WALLS = ((-0.03, 0.0, 1.05), (0.08, 0.0, 0.97))


@pytest.mark.parametrize("prec,rec", PRECS, ids=PID)
@pytest.mark.parametrize("nx,ny,bcx", [(70, 37, 0), (262, 40, 1), (33, 9, 1), (130, 3, 0)])
def test_step_2d_walls_parity(prec, rec, nx, ny, bcx):
    """Moving, heated walls below row 0 and above row ny-1 by non-equilibrium
    extrapolation, on a sheared reactive non-equilibrium state: several strips and tiles,
    ragged edges, and grids thinner than the ghost rows (ny = 3)."""
    params, fields = mixed_2d(nx, ny, bc=(bcx, 2), seed=nx + 1)
    params["walls"] = WALLS
    s, ob, f, lam = start(params, fields, prec, rec, noise_seed=ny + 1)
    steps = 25
    s.step(steps)
    f_ref, lam_ref = ob.run(f, lam, steps)
    got = s.f_planes()
    for i in range(16):
        assert rel_l2(got[i], f_ref[i]) <= TOL[prec], ("f", i + 1, rel_l2(got[i], f_ref[i]))
    assert rel_l2(got[16], lam_ref) <= TOL[prec]
    m, mr = s.macros(), ob.macros(f_ref)
    for k in ("rho", "ux", "uy", "T", "p"):
        assert rel_l2(m[k], mr[k]) <= TOL[prec], (k, rel_l2(m[k], mr[k]))


SIDES = {
    # Dirichlet inflow at x = 0, outflow at x = nx, specular floor, Dirichlet lid
    "inflow": ((3, 1.05, 0.15, 0.0, 1.1, 0.2), (1, 1, 0, 0, 1, 0),
               (4, 1, 0, 0, 1, 0), (3, 0.95, 0.1, -0.05, 1.15, 0.3)),
    # outflow at x = 0, Dirichlet at x = nx, a moving heated wall below, specular above
    "mixed": ((1, 1, 0, 0, 1, 0), (3, 0.9, -0.1, 0.02, 1.2, 0.1),
              (2, 1, 0, 0, 1, 0), (4, 1, 0, 0, 1, 0)),
}


@pytest.mark.parametrize("prec,rec", PRECS, ids=PID)
@pytest.mark.parametrize("kind", ["inflow", "mixed"])
@pytest.mark.parametrize("nx,ny", [(70, 37), (262, 40), (33, 9), (130, 3)])
def test_step_2d_per_side_parity(prec, rec, kind, nx, ny):
    """Per-side conditions (Sec. IV.C): Dirichlet equilibria, specular reflection,
    zero-gradient outflow and a non-equilibrium-extrapolation wall, on a sheared
    reactive non-equilibrium state."""
    params, fields = mixed_2d(nx, ny, bc=(5, 5), seed=nx + 2)
    params["sides"] = SIDES[kind]
    params["walls"] = WALLS
    s, ob, f, lam = start(params, fields, prec, rec, noise_seed=ny + 2)
    steps = 25
    s.step(steps)
    f_ref, lam_ref = ob.run(f, lam, steps)
    got = s.f_planes()
    for i in range(16):
        assert rel_l2(got[i], f_ref[i]) <= TOL[prec], ("f", i + 1, rel_l2(got[i], f_ref[i]))
    assert rel_l2(got[16], lam_ref) <= TOL[prec]
    m, mr = s.macros(), ob.macros(f_ref)
    for k in ("rho", "ux", "uy", "T", "p"):
        assert rel_l2(m[k], mr[k]) <= TOL[prec], (k, rel_l2(m[k], mr[k]))


def test_shock_reflection_parity_and_incident_shock():
    """Shock reflection set-up of Sec. IV.C on the paper's 300 x 100 grid: the CUDA FP64
    and FP32 runs against the oracle after 2000 steps, then to t = 0.08 on the GPU,
    where the incident shock (between the inflow state and the lid's post-shock state,
    Mach 2.3094) must stand at the 30 degrees the Rankine-Hugoniot relations give: the
    level rho = 1.125 crossed at y = H - x tan(phi), fitted over x in [0.02, 0.09]
    (the oracle gives 29.7 degrees there; the shock bends near the corner it starts
    from). Past t ~ 0.11 the 16-velocity model with this table goes unstable behind the
    reflection, in the oracle as on the GPU, so the reflected state is not checked."""
    c = li.shock_reflection(steps=2000)
    p, fl = c["params"], c["fields"]
    ob = make_oracle(p)
    f0 = ob.init(fl["rho"], fl["ux"], fl["uy"], fl["T"])
    f_ref, lam_ref = ob.run(f0, fl["lam"], c["steps"])
    mr = ob.macros(f_ref)
    # the Mach-2.3 shock amplifies rounding-size differences (measured 4e-9 after 2000
    # steps between the CUDA FP64 run and the oracle): bound FP64 by the oracle's own
    # drift under a 1e-15 perturbation
    rng = np.random.default_rng(li.SEED_BASE + 19)
    fp, _ = ob.run(f0 * (1 + 1e-15 * rng.standard_normal(f0.shape)), fl["lam"], c["steps"])
    mp = ob.macros(fp)
    ny, nx, dx = p["ny"], p["nx"], p["dx"]
    for prec in (lbkm.F64, lbkm.F32):
        s = solver(p, prec)
        s.init_fields(fl["rho"], fl["ux"], fl["uy"], fl["T"], fl["lam"])
        s.step(c["steps"])
        m = s.macros()
        # FP32: the uniform inflow recomputes its equilibrium every step (S dt up to 1)
        # and its rounding repeats identically, drifting linearly (2.9e-4 in rho after
        # 2000 steps), so FP32 is held to 1e-3 here (u_y, nonzero only behind the
        # shock, to 5e-3 of its smaller norm; 2.7e-3 measured)
        for k in ("rho", "ux", "uy", "T"):
            tol = (max(1e-12, 20 * rel_l2(mp[k], mr[k])) if prec == lbkm.F64
                   else (5e-3 if k == "uy" else 1e-3))
            assert rel_l2(m[k], mr[k]) <= tol, (prec, k, rel_l2(m[k], mr[k]), tol)
        s.step(16000 - c["steps"])
        rho = s.macros()["rho"]
        ys = (np.arange(ny) + 0.5) * dx
        xs, yshock = [], []
        for j in range(20, 90, 5):
            col = rho[:, j]
            i = int(np.where(col > 1.125)[0].min())
            yshock.append(ys[i - 1] + (1.125 - col[i - 1]) * dx / (col[i] - col[i - 1]))
            xs.append((j + 0.5) * dx)
        slope = np.polyfit(xs, yshock, 1)[0]
        angle = np.degrees(np.arctan(-slope))
        assert abs(angle - 30.0) < 1.5, (prec, angle)
        behind = rho[-8:-3, 30:60].mean()  # between the shock and the lid
        assert abs(behind / 1.25 - 1) < 0.02, (prec, behind)


@pytest.mark.parametrize("prec", [lbkm.F64, lbkm.F32], ids=["f64", "f32"])
def test_couette_full_run(prec):
    """Couette start-up (Sec. IV.D, 200 rows, t = 0.5): every field against the oracle
    at 1000 steps to the plain tolerance, and at the end the velocity profile against
    the series solution no worse than the oracle's (FP32 within 10 %)."""
    c = li.couette()
    p, fl = c["params"], c["fields"]
    s = solver(p, prec)
    s.init_fields(fl["rho"], fl["ux"], fl["uy"], fl["T"], fl["lam"])
    ob = make_oracle(p)
    f0 = ob.init(fl["rho"], fl["ux"], fl["uy"], fl["T"])
    if prec == lbkm.F32:
        f0 = f0.astype(np.float32).astype(np.float64)
    s.step(1000)
    f, lam = ob.run(f0, fl["lam"], 1000)
    m, mr = s.macros(), ob.macros(f)
    for k in ("rho", "ux", "T", "p"):
        assert rel_l2(m[k], mr[k]) <= TOL[prec], (k, rel_l2(m[k], mr[k]))
    s.step(c["steps"] - 1000)
    f, lam = ob.run(f, lam, c["steps"] - 1000)
    m, mr = s.macros(), ob.macros(f)
    assert rel_l2(m["ux"], mr["ux"]) <= (1e-10 if prec == lbkm.F64 else 1e-3)
    ny, dy, u0 = p["ny"], p["dx"], c["u0"]
    H, t, nu = ny * dy, c["steps"] * p["dt"], 1.0 / p["S"][5]
    y = (np.arange(ny) + 0.5) * dy
    ua = u0 * y / H + (2.0 / np.pi) * u0 * sum(
        (-1) ** n / n * np.exp(-(n * np.pi) ** 2 * nu * t / H ** 2) * np.sin(n * np.pi * y / H)
        for n in range(1, 400))
    d_gpu = np.abs(m["ux"][:, 0] - ua).mean()
    d_orc = np.abs(mr["ux"][:, 0] - ua).mean()
    assert d_gpu <= (1.10 if prec == lbkm.F32 else 1.0 + 1e-6) * d_orc, (d_gpu, d_orc)


# ------------------------------------------------------------------ Sod tube and detonation
@pytest.mark.parametrize("run", ["A", "B"])
def test_riemann_full_config_fp64(run):
    c = li.riemann(nx=400, steps=1000, run=run, interface=200)
    fl = c["fields"]
    s = solver(c["params"], lbkm.F64)
    s.init_fields(fl["rho"], fl["ux"], fl["uy"], fl["T"], fl["lam"])
    s.step(c["steps"])
    ob = make_oracle(c["params"])
    f, lam = ob.run(ob.init(fl["rho"], fl["ux"], fl["uy"], fl["T"]), fl["lam"], c["steps"])
    m, mr = s.macros(), ob.macros(f)
    for k in ("rho", "ux", "T", "p"):
        assert rel_l2(m[k], mr[k]) <= 1e-12, (k, rel_l2(m[k], mr[k]))
    assert rel_l2(s.f_planes()[:16], f) <= 1e-12


@pytest.mark.parametrize("which", ["lax", "sjogreen"])
@pytest.mark.parametrize("prec", [lbkm.F64, lbkm.F32], ids=["f64", "f32"])
def test_lax_sjogreen_full_runs(which, prec):
    """Lax (15000 steps, I = 1) and Sjogreen (1500 steps, I = 4) shock tubes of Sec. IV.B,
    every field against the oracle: at an early horizon (before perturbations grow) to
    the plain tolerance, and at the paper's end time to the larger of that tolerance and
    a multiple of the oracle's own drift under a perturbation of the size of one
    rounding of the precision (1e-15 for FP64, 1e-7 for FP32). Both problems amplify
    such perturbations (Sjogreen's near-vacuum centre most: 1e-7 grows to ~3e-3), so the
    end-time comparison is only as sharp as the problem allows."""
    c = getattr(li, which)()
    fl = c["fields"]
    early = {"lax": 1000, "sjogreen": 200}[which]
    s = solver(c["params"], prec)
    s.init_fields(fl["rho"], fl["ux"], fl["uy"], fl["T"], fl["lam"])
    ob = make_oracle(c["params"])
    f0 = ob.init(fl["rho"], fl["ux"], fl["uy"], fl["T"])
    if prec == lbkm.F32:  # the FP32 run starts from the FP32-rounded state
        f0 = f0.astype(np.float32).astype(np.float64)
    tol = TOL[prec]
    s.step(early)
    f, lam = ob.run(f0, fl["lam"], early)
    m, mr = s.macros(), ob.macros(f)
    for k in ("rho", "ux", "T", "p"):
        assert rel_l2(m[k], mr[k]) <= tol, (early, k, rel_l2(m[k], mr[k]))
    assert rel_l2(s.f_planes()[:16], f) <= tol
    s.step(c["steps"] - early)
    f, lam = ob.run(f, lam, c["steps"] - early)
    eps, mult = (1e-15, 20.0) if prec == lbkm.F64 else (1e-7, 4.0)
    rng = np.random.default_rng(li.SEED_BASE + 17)
    fp, _ = ob.run(f0 * (1.0 + eps * rng.standard_normal(f0.shape)), fl["lam"], c["steps"])
    m, mr, mp = s.macros(), ob.macros(f), ob.macros(fp)
    # FP32 arithmetic recomputes the equilibrium every step (S dt = 1 here); in the
    # uniform regions its rounding repeats identically from step to step and so adds up
    # linearly (Lax: 2.5e-4 in rho after 15000 steps), which no perturbation of the
    # initial state reproduces. The FP32 end state is therefore held to 1e-3, and its
    # distance from the exact Euler solution to within 10 % (Lax) or 30 % (Sjogreen,
    # whose centre amplifies 1e-7 to 3e-3) of the oracle's; measured: Lax u +3.9 %,
    # Sjogreen rho +3.5 %, p +20 %. FP64 matches the oracle's distance.
    drift = 1e-3 if prec == lbkm.F32 else 0.0
    for k in ("rho", "ux", "T", "p"):
        bound = max(tol, drift, mult * rel_l2(mp[k], mr[k]))
        assert rel_l2(m[k], mr[k]) <= bound, (k, rel_l2(m[k], mr[k]), bound)
    bound = max(tol, drift, mult * rel_l2(fp, f))
    assert rel_l2(s.f_planes()[:16], f) <= bound, (rel_l2(s.f_planes()[:16], f), bound)
    p = c["params"]
    x = (np.arange(p["nx"]) + 0.5) * p["dx"] - 0.5 * p["nx"] * p["dx"]
    (rl, tl, ul), (rr, tr, ur) = c["left"], c["right"]
    r, u, pe = er.sample((rl, ul, rl * tl), (rr, ur, rr * tr), p["gamma"],
                         x / (c["steps"] * p["dt"]))
    for k, ex in (("rho", r), ("ux", u), ("p", pe)):
        d_gpu, d_orc = np.abs(m[k][0] - ex).mean(), np.abs(mr[k][0] - ex).mean()
        slack = (1.10 if which == "lax" else 1.30) if prec == lbkm.F32 else 1.0 + 1e-6
        assert d_gpu <= slack * d_orc, (k, d_gpu, d_orc)


@pytest.fixture(scope="module")
def detonation_ref():
    """Oracle run of the full 1-D detonation (16384 cells), kept at 2000 and 20000 steps,
    and two references for the long run:
    * the oracle's own spread at 20000 steps: the same run from an initial f perturbed by
      1e-15 (relative). The ignition switch T > T_ig is a hard threshold, so rounding
      differences of that size grow to ~1e-6 over 20000 steps whatever the
      implementation; that spread, not 1e-12, is the attainable FP64 bound there;
    * the cost of FP32 storage alone: the oracle run from the FP32-rounded start with its
      state rounded to FP32 after every step (FP64 arithmetic), per field at 20000 steps.
      The FP32 kernel adds FP32 arithmetic of the same order to that rounding, so its
      bound is four times this figure (or 2e-5 where that is larger)."""
    c = li.detonation(nx=16384, steps=20000)
    fl = c["fields"]
    ob = make_oracle(c["params"])
    f0 = ob.init(fl["rho"], fl["ux"], fl["uy"], fl["T"])
    f1, l1 = ob.run(f0, fl["lam"], 2000)
    f2, l2 = ob.run(f1, l1, 18000)
    fp = f0 * (1 + 1e-15 * np.random.default_rng(0).standard_normal(f0.shape))
    fp, lp = ob.run(fp, fl["lam"], 20000)
    m2, mp = ob.macros(f2), ob.macros(fp)
    spread = {k: rel_l2(mp[k], m2[k]) for k in ("rho", "ux", "T", "p")}
    spread["lam"] = rel_l2(lp, l2)
    f32 = lambda a: np.asarray(a).astype(np.float32).astype(np.float64)
    fs, ls = f32(f0), f32(fl["lam"])
    for _ in range(20000):
        fs, ls = ob.run(fs, ls, 1)
        fs, ls = f32(fs), f32(ls)
    ms = ob.macros(fs)
    storage = {k: rel_l2(ms[k], m2[k]) for k in ("rho", "ux", "T", "p")}
    storage["lam"] = rel_l2(ls, l2)
    return c, ob, {2000: (f1, l1), 20000: (f2, l2)}, spread, storage


@pytest.mark.parametrize("prec,rec", PRECS, ids=PID)
@pytest.mark.parametrize("steps", [2000, 20000])
def test_detonation_full_config(detonation_ref, prec, rec, steps):
    c, ob, ref, spread, storage = detonation_ref
    fl = c["fields"]
    s = solver(c["params"], prec, rec)
    s.init_fields(fl["rho"], fl["ux"], fl["uy"], fl["T"], fl["lam"])
    s.step(steps)
    f, lam = ref[steps]
    m, mr = s.macros(), ob.macros(f)
    errs = {k: rel_l2(m[k], mr[k]) for k in ("rho", "ux", "T", "p")}
    errs["lam"] = rel_l2(m["lam"], lam)
    meets = {k: e <= TOL[prec] for k, e in errs.items()}
    print("detonation", steps, "prec", prec, rec, errs, "oracle spread", spread,
          "FP32 storage alone", storage, "meets the stated tolerance", meets)
    for k, e in errs.items():
        tol = TOL[prec]
        if steps == 20000:
            # past the ignition-switch events the bound is the oracle's own spread
            # (FP64), or four times the cost of FP32 storage (FP32)
            tol = max(tol, 20 * spread[k]) if prec == lbkm.F64 else max(tol, 4 * storage[k])
        assert e <= tol, (k, e, tol)


# ------------------------------------------------------------------ single relaxation time
@pytest.mark.parametrize("rec", [0, 1], ids=["f32", "f32-df"])
@pytest.mark.parametrize("nx,ny,bc", [(300, 77, (0, 0)), (262, 40, (1, 1)), (45, 19, (1, 0))])
def test_srt_fast_path_matches_oracle_and_moment_form(rec, nx, ny, bc):
    """Equal rates R_5..R_16 without TNE select the single-relaxation-time kernel (Sec. V,
    Eq. (87): -S (f - f^eq) + C in velocity space, no forward transform): against the
    oracle's moment-space step, whose BGK limit it is (relative L2 <= 2e-5 per field), and
    against the moment-space kernel forced by collision = 1 (rounding differences only)."""
    params, fields = mixed_2d(nx, ny, bc=bc, seed=nx)
    params = dict(params, S=np.full(16, 6e4))
    steps = 20
    s, ob, f, lam = start(params, fields, lbkm.F32, rec, noise_seed=ny)
    m_, _, _, _ = start(params, fields, lbkm.F32, rec, noise_seed=ny, collision=1)
    s.step(steps)
    m_.step(steps)
    f_ref, lam_ref = ob.run(f, lam, steps)
    got, mrt = s.f_planes(), m_.f_planes()
    for i in range(16):
        assert rel_l2(got[i], f_ref[i]) <= TOL[lbkm.F32], ("f", i + 1)
        assert rel_l2(got[i], mrt[i]) <= 1e-5, ("vs moment form", i + 1)
    assert rel_l2(got[16], lam_ref) <= TOL[lbkm.F32]
    s.close()
    m_.close()


# ------------------------------------------------------------------ caller-owned memory
def test_torch_allocator_owns_every_buffer():
    """lbkm_params.alloc / free backed by torch's caching allocator: the handle, its
    temporaries (macros to host) and lbkm_tne's fields come from torch tensors, and the
    results are bitwise those of a handle that allocates for itself."""
    import torch
    params, fields = mixed_2d(130, 37, bc=(0, 0), seed=4)
    talloc = lbkm.TorchAllocator()
    before = torch.cuda.memory_allocated()
    a, ob, f, lam = start(params, fields, lbkm.F32, 0, noise_seed=2, allocator=talloc,
                          tne_every=1, tne_capacity=4)
    n_create = talloc.allocated
    assert n_create >= 6 and torch.cuda.memory_allocated() > before
    b, _, _, _ = start(params, fields, lbkm.F32, 0, noise_seed=2, tne_every=1, tne_capacity=4)
    for s in (a, b):
        s.step(7)
    ma, mb = a.macros(), b.macros()
    assert talloc.allocated > n_create  # the host copy of the macros used a torch block
    for k in ma:
        assert np.array_equal(ma[k], mb[k]), k
    assert np.array_equal(a.f_planes(), b.f_planes())
    da, ga = a.tne(fields=True)
    db, gb = b.tne(fields=True)
    assert np.array_equal(da, db) and np.array_equal(ga["sum"], gb["sum"])
    live = len(talloc.blocks)
    a.close()
    b.close()
    assert len(talloc.blocks) == 0 < live  # every block went back through free


# ------------------------------------------------------------------ config 3 at length
@pytest.fixture(scope="module")
def reactive_window_ref():
    """The oracle on a periodic 1024 x 1024 window of the 2-D reactive-field recipe for its
    full 500 steps from the FP32-rounded start (with the TNE record of every step), and the
    same run with its state rounded to FP32 after every step (FP64 arithmetic): the cost
    of FP32 storage alone, per plane."""
    return _storage_ref(li.reactive2d(n=1024, steps=500))


def _storage_ref(c):
    fl = c["fields"]
    ob = make_oracle(c["params"])
    f32 = lambda a: np.asarray(a).astype(np.float32).astype(np.float64)
    f0 = f32(ob.init(fl["rho"], fl["ux"], fl["uy"], fl["T"]))
    l0 = f32(fl["lam"])
    f_ref, lam_ref, hist = ob.run(f0, l0, c["steps"], tne=True)
    fs, ls = f0, l0
    for _ in range(c["steps"]):
        fs, ls = ob.run(fs, ls, 1)
        fs, ls = f32(fs), f32(ls)
    storage = [rel_l2(fs[i], f_ref[i]) for i in range(16)] + [rel_l2(ls, lam_ref)]
    return c, ob, f0, l0, f_ref, lam_ref, hist, storage


@pytest.mark.parametrize("prec,rec", [(lbkm.F32, 0), (lbkm.F32, 1)], ids=["f32", "f32-df"])
def test_reactive2d_window_full_length(reactive_window_ref, prec, rec):
    """A periodic 1024 x 1024 window of the 2-D reactive-field recipe for its full 500
    steps, every plane compared element by element with the oracle, with the TNE record
    of every step. The bound per plane is the larger of 2e-5 and twice the cost of FP32
    storage alone (the kernel adds FP32 arithmetic to that rounding). The grid has 512
    strips of 16 rows for 304 resident blocks, so the persistent strip loop wraps."""
    c, ob, f0, l0, f_ref, lam_ref, hist, storage = reactive_window_ref
    s = solver(c["params"], prec, rec, tne_every=1, tne_capacity=500)
    s.set_state(state_bytes(np.concatenate([f0, l0[None]]), prec))
    s.step(c["steps"])
    got = s.f_planes()
    errs = [rel_l2(got[i], f_ref[i]) for i in range(16)] + [rel_l2(got[16], lam_ref)]
    print("reactive2d 1024^2 x 500: plane errors", np.round(np.array(errs) / 1e-5, 2).tolist(),
          "x1e-5; FP32 storage alone", np.round(np.array(storage) / 1e-5, 2).tolist(), "x1e-5")
    for i, e in enumerate(errs):
        assert e <= max(2e-5, 2 * storage[i]), (i, e, storage[i])
    m, mr = s.macros(), ob.macros(f_ref)
    merr = {k: rel_l2(m[k], mr[k]) for k in ("rho", "ux", "uy", "T", "p")}
    print("reactive2d 1024^2 x 500: macro errors", merr)
    for k, e in merr.items():
        assert e <= max(2e-5, 2 * max(storage)), k
    recs = s.tne_history()
    assert len(recs) == c["steps"]
    # record scales as in test_tne_fields_and_on_the_fly_records (Delta_k cancels digits
    # of f_hat_k); at step 0 both sides see the same state (tolerance 2e-5), later the
    # states themselves differ by up to the bound above, so the records by twice that
    area = c["params"]["dx"] ** 2
    fh = np.abs(np.einsum("ki,iyx->kyx", ob.M, f0))
    sscale, dscale = fh.sum(axis=(1, 2)) * area, np.sqrt((fh[4:] ** 2).sum(axis=0)).sum() * area
    for n in (0, 250, 499):
        want = oracle_unpack(hist[n])
        tol = 2e-5 if n == 0 else 2 * max(2e-5, 2 * max(storage))
        assert np.all(np.abs(recs[n]["sum"] - want["sum"]) <= tol * sscale), n
        assert np.all(np.abs(recs[n]["abs_sum"] - want["abs_sum"]) <= tol * sscale), n
        assert abs(recs[n]["d_sum"] - want["d_sum"]) <= tol * dscale, n


@pytest.fixture(scope="module")
def wrapping_strips_ref():
    """The oracle on a periodic 2310 x 1050 field of the same recipe, 100 steps, and the
    same run with its state rounded to FP32 after every step."""
    return _storage_ref(li.reactive2d(n=2310, ny=1050, steps=100))


@pytest.mark.parametrize("prec,rec", [(lbkm.F32, 0), (lbkm.F32, 1)], ids=["f32", "f32-df"])
def test_reactive2d_strips_of_the_bench_wrap(wrapping_strips_ref, prec, rec):
    """The strip shape the bench runs (64 rows x 128 columns) on a grid of 19 x 17 = 323
    strips for 304 resident blocks, so the persistent strip loop wraps; a 6-column strip
    at the x edge and a 26-row strip at the y edge; 100 steps against the oracle, every
    plane element by element, bound as in the 1024 x 1024 window test."""
    c, ob, f0, l0, f_ref, lam_ref, hist, storage = wrapping_strips_ref
    s = solver(c["params"], prec, rec, tne_every=1, tne_capacity=100)
    s.set_state(state_bytes(np.concatenate([f0, l0[None]]), prec))
    s.step(c["steps"])
    got = s.f_planes()
    errs = [rel_l2(got[i], f_ref[i]) for i in range(16)] + [rel_l2(got[16], lam_ref)]
    print("reactive2d 2310x1050 x 100: plane errors", np.round(np.array(errs) / 1e-5, 2).tolist(),
          "x1e-5; FP32 storage alone", np.round(np.array(storage) / 1e-5, 2).tolist(), "x1e-5")
    for i, e in enumerate(errs):
        assert e <= max(2e-5, 2 * storage[i]), (i, e, storage[i])
    recs = s.tne_history()
    assert [r["step"] for r in recs] == list(range(c["steps"]))
    area = c["params"]["dx"] ** 2
    fh = np.abs(np.einsum("ki,iyx->kyx", ob.M, f0))
    sscale = fh.sum(axis=(1, 2)) * area
    for n in (0, 99):
        want = oracle_unpack(hist[n])
        tol = 2e-5 if n == 0 else 2 * max(2e-5, 2 * max(storage))
        assert np.all(np.abs(recs[n]["abs_sum"] - want["abs_sum"]) <= tol * sscale), n
    s.close()


# ------------------------------------------------------------------ full 2-D size, sampled
@pytest.mark.parametrize("prec,rec", [(lbkm.F32, 0), (lbkm.F32, 1)], ids=["f32", "f32-df"])
def test_reactive2d_full_size_sampled(prec, rec):
    """4096 x 4096 periodic reactive field, 3 steps in the bench's configuration (TNE every
    step): sampled cells against the oracle run on a periodic patch around each sample
    (the update has radius 2 per step)."""
    import torch
    c = li.reactive2d(n=4096, steps=3)
    fl = c["fields"]
    s = solver(c["params"], prec, rec, tne_every=1, tne_capacity=4)
    s.init_fields(fl["rho"], fl["ux"], fl["uy"], fl["T"], fl["lam"])
    steps = c["steps"]
    s.step(steps)
    planes = s.planes_device()
    n = 4096
    rng = np.random.default_rng(42)
    samples = [(0, 0), (n - 1, n - 1), (0, n - 1), (n - 1, 0), (1, 2)] + [
        tuple(rng.integers(0, n, 2)) for _ in range(15)]
    R = 2 * steps + 2
    p = dict(c["params"])
    p.update(nx=2 * R + 1, ny=2 * R + 1, bc_x=1, bc_y=1)
    ob = make_oracle(p)
    for (yy, xx) in samples:
        iy = np.arange(yy - R, yy + R + 1) % n
        ix = np.arange(xx - R, xx + R + 1) % n
        patch = {k: fl[k][np.ix_(iy, ix)] for k in fl}
        f = ob.init(patch["rho"], patch["ux"], patch["uy"], patch["T"])
        f, lam = ob.run(f, patch["lam"], steps)
        want = np.concatenate([f[:, R, R], [lam[R, R]]])
        got = planes[:, yy, xx].double().cpu().numpy()
        assert np.abs(got - want).max() <= 2e-5 * np.abs(want).max(), (yy, xx)
    del torch


@pytest.mark.parametrize("rec", [0, 1], ids=["f32", "f32-df"])
def test_reactive2d_full_size_tne_record(rec):
    """The bench's workload at full size (4096 x 4096, TNE every step): the on-the-fly record
    of step 2 against the oracle's record of the very state the kernel stepped there, read
    back, within the FP32-arithmetic bound of test_tne_record_within_the_fp32_arithmetic_bound
    (per cell |dDelta_k| <= 16 u S_k; exact sums)."""
    u = 2.0 ** -24
    c = li.reactive2d(n=4096, steps=3)
    fl = c["fields"]
    s = solver(c["params"], lbkm.F32, rec, tne_every=1, tne_capacity=4)
    s.init_fields(fl["rho"], fl["ux"], fl["uy"], fl["T"], fl["lam"])
    s.step(2)
    fs = s.f_planes()[:16]
    s.step(1)
    h = s.tne_history()[-1]
    assert h["step"] == 2
    s.close()
    ob = make_oracle(c["params"])
    delta, r = ob.tne(fs, fields=True)
    area = c["params"]["dx"] ** 2
    fh = np.einsum("ki,iyx->kyx", ob.M, fs)
    S = np.einsum("ki,iyx->kyx", np.abs(ob.M), np.abs(fs))
    S += np.abs(fh - delta)
    E = 16 * u * S[4:]
    del fh, S
    for key, b in (("sum", area * E.sum(axis=(1, 2))), ("abs_sum", area * E.sum(axis=(1, 2))),
                   ("min", E.max(axis=(1, 2))), ("max", E.max(axis=(1, 2)))):
        err = np.abs(np.asarray(h[key])[4:] - np.asarray(r[key])[4:])
        assert np.all(err <= b), (key, float(np.max(err / b)))
    d = np.sqrt((delta[4:] ** 2).sum(axis=0))
    bd = area * (np.sqrt((E ** 2).sum(axis=0)) + (8 + 31) * u * d).sum()
    assert abs(h["d_sum"] - r["d_sum"]) <= bd


# ------------------------------------------------------------------ TNE
@pytest.mark.parametrize("prec,rec", PRECS, ids=PID)
def test_tne_fields_and_on_the_fly_records(prec, rec):
    params, fields = mixed_2d(40, 17, seed=3)
    steps = 6
    s, ob, f, lam = start(params, fields, prec, rec, noise_seed=5, tne_every=1, tne_capacity=16)
    s.step(steps)
    hist = s.tne_history()
    assert [h["step"] for h in hist] == list(range(steps))
    fs, ls = f, lam
    area = params["dx"] * params["dx"]
    for k in range(steps):
        _, rec_ref = ob.tne(fs, fields=False)
        h = hist[k]
        # Delta_k = f_hat_k - f_hat^eq_k cancels several digits, so its rounding error
        # scales with |f_hat_k|, the magnitude of the moments it is taken from
        fh = np.abs(np.einsum("ki,iyx->kyx", ob.M, fs))
        tol = 1e-12 if prec == lbkm.F64 else 2e-5
        sscale = fh.sum(axis=(1, 2)) * area
        mscale = fh.max(axis=(1, 2))
        assert np.all(np.abs(h["sum"] - rec_ref["sum"]) <= tol * sscale), k
        assert np.all(np.abs(h["abs_sum"] - rec_ref["abs_sum"]) <= tol * sscale), k
        assert np.all(np.abs(h["min"] - rec_ref["min"]) <= tol * mscale), k
        assert np.all(np.abs(h["max"] - rec_ref["max"]) <= tol * mscale), k
        dscale = np.sqrt((fh[4:] ** 2).sum(axis=0)).sum() * area
        assert abs(h["d_sum"] - rec_ref["d_sum"]) <= tol * dscale
        assert abs(h["d2_sum"] - rec_ref["d2_sum"]) <= tol * dscale * mscale[4:].max()
        fs, ls = ob.step(fs, ls)
    # lbkm_tne on the current state (FP64 arithmetic on the stored state)
    delta, g = s.tne(fields=True)
    cur = s.f_planes()[:16]
    dref, gref = ob.tne(cur)
    assert np.abs(delta - dref).max() <= 1e-12 * np.abs(dref).max()
    assert np.abs(g["abs_sum"] - gref["abs_sum"]).max() <= 1e-12 * gref["abs_sum"].max()
    assert np.all(delta[:4] == 0)


@pytest.mark.parametrize("rec", [0, 1], ids=["f32", "f32-df"])
@pytest.mark.parametrize("nx,ny", [(300, 140), (1030, 261)])
def test_tne_record_within_the_fp32_arithmetic_bound(rec, nx, ny):
    """The FP32 step kernel's on-the-fly TNE record (Sec. VI, Eqs. (90)-(91)) against the
    oracle's record of the very state the kernel stepped (read back before each step), so
    no trajectory difference enters. What is left is the FP32 arithmetic of each cell's
    Delta_k = f_hat_k - f_hat^eq_k and the summation. A moment passes at most seven
    rounded operations (two butterfly levels, a four-term dot product, one more sum), an
    equilibrium moment at most eight from the FP32-rounded macros (its terms share one
    sign), the difference one more, so per cell |dDelta_k| <= 16 u S_k with u = 2^-24
    and S_k = sum_i |M_ki| |f_i| + |f_hat^eq_k|.
    The sums of Delta_k and |Delta_k| over cells are exact (each thread's FP32 sums carry
    their rounding errors; everything past the thread is FP64), so they may differ from
    the oracle's by no more than the sums of those per-cell bounds; the one-signed sums of
    d and d^2 add at most 31 u of themselves (FP32 over 32 terms per column)."""
    u = 2.0 ** -24
    params, fields = mixed_2d(nx, ny, seed=nx + ny)
    s, ob, f, lam = start(params, fields, lbkm.F32, rec, noise_seed=7, tne_every=1,
                          tne_capacity=8)
    area = params["dx"] * params["dx"]
    absM = np.abs(ob.M)
    worst = {}
    for k in range(3):
        fs = s.f_planes()[:16]
        s.step(1)
        h = s.tne_history()[-1]
        assert h["step"] == k
        delta, r = ob.tne(fs, fields=True)
        fh = np.einsum("ki,iyx->kyx", ob.M, fs)
        S = (np.einsum("ki,iyx->kyx", absM, np.abs(fs)) + np.abs(fh - delta))[4:]
        E = 16 * u * S
        D = delta[4:]
        d = np.sqrt((D ** 2).sum(axis=0))
        bound = dict(
            sum=area * E.sum(axis=(1, 2)), abs_sum=area * E.sum(axis=(1, 2)),
            min=E.max(axis=(1, 2)), max=E.max(axis=(1, 2)),
            # d: the per-cell bound on the vector of errors, the FP32 accumulation of
            # twelve squares and the hardware square root (relative 2^-23)
            d_sum=area * (np.sqrt((E ** 2).sum(axis=0)) + (8 + 31) * u * d).sum(),
            d2_sum=area * ((2 * np.abs(D) * E + E ** 2).sum(axis=0) + (12 + 31) * u * d ** 2).sum())
        for key, b in bound.items():
            got, want = np.asarray(h[key], float), np.asarray(r[key], float)
            if got.ndim:  # index k - 1 holds Delta_k; Delta_1..4 vanish
                got, want = got[4:], want[4:]
            err = np.abs(got - want)
            ratio = float(np.max(err / b))
            worst[key] = max(worst.get(key, 0.0), ratio)
            assert ratio <= 1.0, (k, key, ratio)
    print("TNE record %dx%d rec %d: error / arithmetic bound" % (nx, ny, rec),
          {k: round(v, 4) for k, v in worst.items()})
    s.close()


# ------------------------------------------------------------------ runtime behaviour
def test_pinned_host_fields_are_used_in_place():
    """init_fields from page-locked host tensors (read by the kernel in place) leaves the
    state init_fields from pageable arrays leaves; macros into page-locked outputs
    (written in place) equal macros into pageable arrays, bit for bit."""
    import torch
    nx, ny = 70, 37
    params, fields = mixed_2d(nx, ny, seed=2)
    names = ("rho", "ux", "uy", "T", "lam")
    a, b = solver(params, lbkm.F32), solver(params, lbkm.F32)
    a.init_fields(*[fields[k] for k in names])
    pinned = [torch.from_numpy(np.array(np.broadcast_to(fields[k], (ny, nx)), np.float64)).pin_memory()
              for k in names]
    b.init_fields(*pinned)
    assert np.array_equal(a.get_state(), b.get_state())
    a.step(5)
    b.step(5)
    want = a.macros()
    outs = {k: torch.full((ny, nx), np.nan, dtype=torch.float64).pin_memory()
            for k in ("rho", "ux", "uy", "T", "p", "lam")}
    b.macros(out=outs)
    for k, t in outs.items():
        assert np.array_equal(t.numpy(), want[k]), k
    a.close()
    b.close()


def test_graph_chunks_equal_single_steps():
    params, fields = mixed_2d(50, 20, seed=9)
    a = solver(params, lbkm.F64, tne_every=3, tne_capacity=64)
    b = solver(params, lbkm.F64, tne_every=3, tne_capacity=64)
    for s in (a, b):
        s.init_fields(fields["rho"], fields["ux"], fields["uy"], fields["T"], fields["lam"])
    a.step(71)  # two 32-step graph replays + 7 single launches
    for _ in range(71):
        b.step(1)
    assert np.array_equal(a.get_state(), b.get_state())
    ha, hb = a.tne_history(), b.tne_history()
    assert len(ha) == 24 and [h["step"] for h in ha] == list(range(0, 71, 3))
    assert all(np.array_equal(x["sum"], y["sum"]) for x, y in zip(ha, hb))


def test_tne_history_ring_keeps_the_newest_records():
    """A history ring of 8 after 20 recorded steps holds steps 12..19, in order and equal
    to those records of a run with room for all of them (the copy wraps at the ring's end)."""
    params, fields = mixed_2d(45, 19, seed=6)
    a = solver(params, lbkm.F32, tne_every=1, tne_capacity=8)
    b = solver(params, lbkm.F32, tne_every=1, tne_capacity=32)
    for s in (a, b):
        s.init_fields(fields["rho"], fields["ux"], fields["uy"], fields["T"], fields["lam"])
        s.step(20)
    ha, hb = a.tne_history(), b.tne_history()
    assert [h["step"] for h in ha] == list(range(12, 20))
    assert [h["step"] for h in hb] == list(range(20))
    for x, y in zip(ha, hb[12:]):
        for k in ("sum", "abs_sum", "min", "max"):
            assert np.array_equal(x[k], y[k]), k
        assert x["d_sum"] == y["d_sum"] and x["d2_sum"] == y["d2_sum"]
    assert [h["step"] for h in a.tne_history(max_records=3)] == [12, 13, 14]
    a.close()
    b.close()


@pytest.mark.parametrize("rec", [0, 1], ids=["f32", "f32-df"])
def test_tne_every_k_matches_every_step_fp32(rec):
    """The FP32 2-D step with tne_every = 3 (statistics gathered every step, reduced on the
    due ones) records steps 0, 3, 6, ... exactly as the run that records every step, and
    leaves the same state; a handle without TNE (the kernel without any TNE code) leaves
    that state too. Ragged strips in x and y."""
    params, fields = mixed_2d(150, 70, seed=12)
    runs = {}
    for k in (1, 3, 0):
        s = solver(params, lbkm.F32, rec, tne_every=k, tne_capacity=16)
        s.init_fields(fields["rho"], fields["ux"], fields["uy"], fields["T"], fields["lam"])
        s.step(10)
        runs[k] = (s.get_state(), s.tne_history() if k else [])
        s.close()
    every, third = runs[1][1], runs[3][1]
    assert [h["step"] for h in third] == [0, 3, 6, 9]
    for h in third:
        g = every[h["step"]]
        for key in ("sum", "abs_sum", "min", "max"):
            assert np.array_equal(h[key], g[key]), (h["step"], key)
        assert h["d_sum"] == g["d_sum"] and h["d2_sum"] == g["d2_sum"]
    assert np.array_equal(runs[3][0], runs[1][0])
    assert np.array_equal(runs[0][0], runs[1][0])


def test_checkpoint_resume_is_bitwise():
    params, fields = mixed_2d(33, 12, seed=4)
    a = solver(params, lbkm.F32)
    a.init_fields(fields["rho"], fields["ux"], fields["uy"], fields["T"], fields["lam"])
    a.step(40)
    mid = a.get_state()
    a.step(40)
    b = solver(params, lbkm.F32)
    b.set_state(mid)
    assert b.steps_taken == 40
    b.step(40)
    assert np.array_equal(a.get_state(), b.get_state())


def test_zero_steps_and_tiny_grids():
    for nx, ny in ((1, 1), (3, 1), (2, 2), (5, 3)):
        params, fields = mixed_2d(nx, ny, bc=(0, 0), seed=nx + ny)
        s, ob, f, lam = start(params, fields, lbkm.F64, 0, noise_seed=1)
        s.step(0)
        assert np.allclose(s.f_planes()[:16], f, rtol=0, atol=0)
        s.step(7)
        f_ref, lam_ref = ob.run(f, lam, 7)
        assert rel_l2(s.f_planes()[:16], f_ref) <= 1e-12, (nx, ny)


def test_nonfinite_state_is_reported():
    params, fields = mixed_2d(20, 4, seed=2)
    s, ob, f, lam = start(params, fields, lbkm.F64, 0)
    f = f.copy()
    f[3, 2, 5] = np.nan
    s.set_state(state_bytes(np.concatenate([f, lam[None]]), lbkm.F64))
    s.step(1)
    with pytest.raises(lbkm.LbkmError) as e:
        s.sync()
    assert e.value.code == 5
