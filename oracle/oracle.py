"""ctypes binding of the plain FP64 C oracle (``lbkm_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
CPU-baseline leg of the benchmark, never by the product path. The binding only
marshals arguments; every step of the model is computed in ``lbkm_oracle.c``.

Model set-up that the oracle needs besides the C code, written here on the
oracle side and shared with nothing:
  * the velocity table of an orbit model: orbits of kind 0 are the axis set
    cyc(+-1, 0), kind 1 the diagonal set (+-1, +-1), each scaled by the orbit
    speed and carrying one eta. Four orbits give the 16-velocity model (the D2V24
    construction of Sec. II, Eqs. (25)-(27), cut to 16 velocities as Sec. VII
    allows); six orbits (axis, diagonal) x (v_a, v_b, v_c) give the paper's D2V24,
    run by the same C source built with 24 velocities (``liboracle24.so``);
  * I from gamma: gamma = (D + I + 2) / (D + I)  (Sec. III, Eq. (68)).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

NV = 16
D = 2
TNE_LEN = 4 * NV + 2
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbkm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIBS = {16: _LIB, 24: os.path.join(_HERE, "liboracle24.so")}

# velocity order inside an orbit: (1,0),(0,1),(-1,0),(0,-1) and
# (1,1),(-1,1),(-1,-1),(1,-1)
_AXIS = [(1, 0), (0, 1), (-1, 0), (0, -1)]
_DIAG = [(1, 1), (-1, 1), (-1, -1), (1, -1)]


def build(force: bool = False, nv: int = 16) -> str:
    """Compile the oracle with nv velocities (16: ``liboracle.so``, 24:
    ``liboracle24.so``) next to its source (gcc, OpenMP)."""
    lib = _LIBS[nv]
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        tmp = lib + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-DNV=%d" % nv, "-o", tmp,
             _SRC, "-lm"]
        )
        os.replace(tmp, lib)
    return lib


def _params_fields(nv):
    return [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("bc_x", ctypes.c_int32), ("bc_y", ctypes.c_int32),
        ("vx", ctypes.c_double * nv), ("vy", ctypes.c_double * nv), ("eta", ctypes.c_double * nv),
        ("I", ctypes.c_double), ("S", ctypes.c_double * nv),
        ("Q", ctypes.c_double), ("omega1", ctypes.c_double), ("omega2", ctypes.c_double),
        ("T_ig", ctypes.c_double),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dt", ctypes.c_double),
        ("wall_ux", ctypes.c_double * 2), ("wall_uy", ctypes.c_double * 2),
        ("wall_T", ctypes.c_double * 2),
        ("side_bc", ctypes.c_int32 * 4), ("side_rho", ctypes.c_double * 4),
        ("side_ux", ctypes.c_double * 4), ("side_uy", ctypes.c_double * 4),
        ("side_T", ctypes.c_double * 4), ("side_lam", ctypes.c_double * 4),
        ("time_scheme", ctypes.c_int32),
    ]


class Params(ctypes.Structure):
    _fields_ = _params_fields(16)


class Params24(ctypes.Structure):
    _fields_ = _params_fields(24)


_PARAMS = {16: Params, 24: Params24}
_libs = {}
_dp = ctypes.POINTER(ctypes.c_double)


def _load(nv: int = 16):
    if nv not in _libs:
        lib = ctypes.CDLL(build(nv=nv))
        P = ctypes.POINTER(_PARAMS[nv])
        lib.orc_build_M.argtypes = [P, _dp]
        lib.orc_invert.argtypes = [_dp, _dp]
        lib.orc_invert.restype = ctypes.c_int
        lib.orc_feq_moments.argtypes = [ctypes.c_double] * 5 + [_dp]
        lib.orc_dfeq_dT.argtypes = [ctypes.c_double] * 5 + [_dp]
        lib.orc_reaction_increment.argtypes = [ctypes.c_double] * 4
        lib.orc_reaction_increment.restype = ctypes.c_double
        lib.orc_init.argtypes = [P, _dp, _dp, _dp, _dp, _dp, _dp]
        lib.orc_macros.argtypes = [P, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        lib.orc_tne.argtypes = [P, _dp, _dp, _dp, _dp]
        lib.orc_step.argtypes = [P, _dp, _dp, _dp, _dp, _dp, _dp]
        lib.orc_step.restype = ctypes.c_int
        lib.orc_run.argtypes = [P, _dp, _dp, _dp, _dp, ctypes.c_int64, _dp]
        lib.orc_run.restype = ctypes.c_int
        lib.orc_nnd_advect_1d.argtypes = [ctypes.c_double, _dp, _dp, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_double, ctypes.c_double]
        _libs[nv] = lib
    return _libs[nv]


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def velocity_table(orbit_kind, orbit_speed, orbit_eta):
    """(vx, vy, eta) of the 4 x (number of orbits) velocities of an orbit model."""
    vx, vy, eta = [], [], []
    for kind, c, e in zip(orbit_kind, orbit_speed, orbit_eta):
        for ux, uy in (_AXIS if kind == 0 else _DIAG):
            vx.append(c * ux)
            vy.append(c * uy)
            eta.append(e)
    return np.array(vx, float), np.array(vy, float), np.array(eta, float)


def I_from_gamma(gamma: float) -> float:
    return 2.0 / (gamma - 1.0) - D


def d2v24_orbits(v, eta):
    """Orbit lists of the paper's D2V24 (Eqs. (25)-(27)) from (v_a, v_b, v_c) and
    (eta_a, eta_b, eta_c): velocities 1-4 axis and 5-8 diagonal at v_a, 9-16 at v_b,
    17-24 at v_c."""
    kinds = [0, 1, 0, 1, 0, 1]
    speeds = [v[0], v[0], v[1], v[1], v[2], v[2]]
    etas = [eta[0], eta[0], eta[1], eta[1], eta[2], eta[2]]
    return kinds, speeds, etas


class Oracle:
    """One model set-up (grid, velocity set, rates, chemistry) with its M and M^-1."""

    def __init__(self, nx, ny, *, gamma, orbit_kind, orbit_speed, orbit_eta, S, Q=0.0,
                 omega1=0.0, omega2=0.0, T_ig=1.1, dx=1e-3, dy=None, dt=1e-5,
                 bc_x=1, bc_y=0, walls=None, sides=None, time_scheme=0):
        nv = 4 * len(orbit_kind)
        if nv not in _PARAMS:
            raise ValueError("4 orbits (16 velocities) or 6 orbits (D2V24)")
        self.nv = nv
        lib = _load(nv)
        p = _PARAMS[nv]()
        p.nx, p.ny, p.bc_x, p.bc_y = int(nx), int(ny), int(bc_x), int(bc_y)
        vx, vy, eta = velocity_table(orbit_kind, orbit_speed, orbit_eta)
        p.vx[:], p.vy[:], p.eta[:] = list(vx), list(vy), list(eta)
        p.I = I_from_gamma(gamma)
        S = np.broadcast_to(np.asarray(S, float), (nv,))
        p.S[:] = list(S)
        p.Q, p.omega1, p.omega2, p.T_ig = float(Q), float(omega1), float(omega2), float(T_ig)
        p.dx, p.dy, p.dt = float(dx), float(dx if dy is None else dy), float(dt)
        if walls is not None:  # ((ux, uy, T) below y = 0, (ux, uy, T) above y = ny)
            for side in (0, 1):
                p.wall_ux[side], p.wall_uy[side], p.wall_T[side] = map(float, walls[side])
        if sides is not None:  # 4 x (code, rho, ux, uy, T, lam): x = 0, x = nx, y = 0, y = ny
            for k, (code, r, u, v, T, lam) in enumerate(sides):
                p.side_bc[k] = int(code)
                p.side_rho[k], p.side_ux[k], p.side_uy[k], p.side_T[k], p.side_lam[k] = (
                    float(r), float(u), float(v), float(T), float(lam))
        p.time_scheme = int(time_scheme)
        self.p = p
        self.nx, self.ny = int(nx), int(ny)
        self.n = self.nx * self.ny
        self.lib = lib
        self.M = np.zeros((nv, nv))
        lib.orc_build_M(ctypes.byref(p), _ptr(self.M))
        self.Minv = np.zeros((nv, nv))
        if lib.orc_invert(_ptr(self.M), _ptr(self.Minv)) != 0:
            raise ValueError("singular moment matrix M for this velocity set")

    # --- model pieces -------------------------------------------------
    def feq_moments(self, rho, ux, uy, T):
        out = np.zeros(self.nv)
        self.lib.orc_feq_moments(rho, ux, uy, T, self.p.I, _ptr(out))
        return out

    def dfeq_dT(self, rho, ux, uy, T):
        out = np.zeros(self.nv)
        self.lib.orc_dfeq_dT(rho, ux, uy, T, self.p.I, _ptr(out))
        return out

    # --- fields ----------------------------------------------------------
    def init(self, rho, ux, uy, T):
        """f = M^-1 f_hat^eq(rho, u, T), shape [nv, ny, nx]."""
        a = [np.ascontiguousarray(np.broadcast_to(np.asarray(v, float), (self.ny, self.nx)))
             for v in (rho, ux, uy, T)]
        f = np.zeros((self.nv, self.ny, self.nx))
        self.lib.orc_init(ctypes.byref(self.p), _ptr(self.Minv), *[_ptr(x) for x in a], _ptr(f))
        return f

    def macros(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = {k: np.zeros((self.ny, self.nx)) for k in ("rho", "ux", "uy", "T", "p")}
        self.lib.orc_macros(ctypes.byref(self.p), _ptr(self.M), _ptr(f), _ptr(out["rho"]),
                           _ptr(out["ux"]), _ptr(out["uy"]), _ptr(out["T"]), _ptr(out["p"]))
        return out

    def tne(self, f, fields=True):
        """(delta [nv, ny, nx] or None, record dict) of a state."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        delta = np.zeros((self.nv, self.ny, self.nx)) if fields else None
        rec = np.zeros(4 * self.nv + 2)
        self.lib.orc_tne(ctypes.byref(self.p), _ptr(self.M), _ptr(f), _ptr(delta), _ptr(rec))
        return delta, unpack_tne(rec)

    def step(self, f, lam):
        f = np.ascontiguousarray(f, dtype=np.float64)
        lam = np.ascontiguousarray(np.broadcast_to(lam, (self.ny, self.nx)), dtype=np.float64)
        fn, ln = np.zeros_like(f), np.zeros_like(lam)
        rc = self.lib.orc_step(ctypes.byref(self.p), _ptr(self.M), _ptr(self.Minv), _ptr(f),
                              _ptr(lam), _ptr(fn), _ptr(ln))
        if rc != 0:
            raise MemoryError("oracle step failed")
        return fn, ln

    def run(self, f, lam, nsteps, tne=False):
        """nsteps steps; returns (f, lam[, tne records of each step's input state])."""
        f = np.array(f, dtype=np.float64, order="C", copy=True)
        lam = np.array(np.broadcast_to(lam, (self.ny, self.nx)), dtype=np.float64, order="C",
                       copy=True)
        hist = np.zeros((int(nsteps), 4 * self.nv + 2)) if tne else None
        rc = self.lib.orc_run(ctypes.byref(self.p), _ptr(self.M), _ptr(self.Minv), _ptr(f),
                             _ptr(lam), int(nsteps), _ptr(hist))
        if rc != 0:
            raise MemoryError("oracle run failed")
        return (f, lam, hist) if tne else (f, lam)


def unpack_tne(rec):
    rec = np.asarray(rec)
    nv = (rec.shape[-1] - 2) // 4
    return {"sum": rec[0:nv].copy(), "abs_sum": rec[nv:2 * nv].copy(),
            "min": rec[2 * nv:3 * nv].copy(), "max": rec[3 * nv:4 * nv].copy(),
            "d_sum": float(rec[4 * nv]), "d2_sum": float(rec[4 * nv + 1])}


def reaction_increment(lam, a, b, dt):
    return _load().orc_reaction_increment(lam, a, b, dt)


def nnd_advect_1d(v, q, dt, dx, bc=0):
    q = np.ascontiguousarray(q, dtype=np.float64)
    out = np.zeros_like(q)
    _load().orc_nnd_advect_1d(v, _ptr(q), _ptr(out), q.size, bc, dt, dx)
    return out
