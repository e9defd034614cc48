"""A second, naive formulation of one MRT-LBKM step, used only to pin the oracle.

It shares nothing with ``oracle/lbkm_oracle.c`` beyond the paper:
  * moments are functions of a continuous (v_x, v_y, eta); M is those functions
    evaluated at the discrete velocities, and M^-1 is never formed (linear solves);
  * f_hat^eq and d f_hat^eq/dT come from Gauss-Hermite quadrature of the
    continuous Maxwellian Eq. (21) and of its T-derivative Eq. (22);
  * collision is the full velocity-space product -M^-1 R_hat M (f - f^eq)
    plus M^-1 A_hat and M^-1 C_hat (Eq. (1) with the sign of A from Eq. (29));
    with 24 velocities (the paper's D2V24, moments m_1..m_24) the chemical term is
    Eq. (24) in velocity space on the quadrature-built f^eq instead;
  * the reaction step integrates Eq. (28) with a library ODE solver;
  * NND is written in its upwind form: for v > 0 the interface value is
    v (f_j + mm(f_j - f_{j-1}, f_{j+1} - f_j)/2), for v < 0
    v (f_{j+1} - mm(f_{j+1} - f_j, f_{j+2} - f_{j+1})/2).
Slow by design: only for grids of a few cells.
"""
from __future__ import annotations

import numpy as np
from scipy.integrate import solve_ivp

D = 2

MOMENTS = [
    lambda vx, vy, e: np.ones_like(vx),
    lambda vx, vy, e: vx,
    lambda vx, vy, e: vy,
    lambda vx, vy, e: vx**2 + vy**2 + e**2,
    lambda vx, vy, e: vx**2,
    lambda vx, vy, e: vx * vy,
    lambda vx, vy, e: vy**2,
    lambda vx, vy, e: (vx**2 + vy**2 + e**2) * vx,
    lambda vx, vy, e: (vx**2 + vy**2 + e**2) * vy,
    lambda vx, vy, e: vx**3,
    lambda vx, vy, e: vx**2 * vy,
    lambda vx, vy, e: vx * vy**2,
    lambda vx, vy, e: vy**3,
    lambda vx, vy, e: (vx**2 + vy**2 + e**2) * vx**2,
    lambda vx, vy, e: (vx**2 + vy**2 + e**2) * vx * vy,
    lambda vx, vy, e: (vx**2 + vy**2 + e**2) * vy**2,
]
# rows m_17..m_24 of the paper's D2V24 (list after Eq. (16))
MOMENTS24 = MOMENTS + [
    lambda vx, vy, e: e**2 * vx**2,
    lambda vx, vy, e: e**2 * vx * vy,
    lambda vx, vy, e: e**2 * vy**2,
    lambda vx, vy, e: (vx**2 + vy**2 + e**2) * e**2,
    lambda vx, vy, e: (vx**2 + vy**2 + e**2) * (vx**2 + vy**2) * vx,
    lambda vx, vy, e: (vx**2 + vy**2 + e**2) * (vx**2 + vy**2) * vy,
    lambda vx, vy, e: (vx**2 + vy**2 + e**2) * e**2 * vx,
    lambda vx, vy, e: (vx**2 + vy**2 + e**2) * e**2 * vy,
]


def _moments(nv):
    return MOMENTS if nv == 16 else MOMENTS24


def maxwellian_moments(rho, ux, uy, T, I, nodes=8, dT=False, nv=16):
    """Moments m_1..m_nv of the continuous f^eq of Eq. (21) (or of df^eq/dT, Eq. (22))."""
    x, w = np.polynomial.hermite_e.hermegauss(nodes)
    w = w / np.sqrt(2.0 * np.pi)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    W = w[:, None, None] * w[None, :, None] * w[None, None, :]
    vx, vy, eta = ux + np.sqrt(T) * X, uy + np.sqrt(T) * Y, np.sqrt(I * T) * Z
    weight = rho * W
    if dT:
        c2 = (vx - ux) ** 2 + (vy - uy) ** 2
        weight = weight * (-(1 + D) * I * T + I * c2 + eta**2) / (2.0 * I * T * T)
    return np.array([np.sum(weight * m(vx, vy, eta)) for m in _moments(nv)])


def velocity_set(orbit_kind, orbit_speed, orbit_eta):
    axis = np.array([[1, 0], [0, 1], [-1, 0], [0, -1]], float)
    diag = np.array([[1, 1], [-1, 1], [-1, -1], [1, -1]], float)
    V, E = [], []
    for k, c, e in zip(orbit_kind, orbit_speed, orbit_eta):
        V.append(c * (axis if k == 0 else diag))
        E.append(np.full(4, e))
    V = np.concatenate(V)
    return V[:, 0], V[:, 1], np.concatenate(E)


def moment_matrix(vx, vy, eta):
    return np.array([m(vx, vy, eta) for m in _moments(len(vx))])


def _mm(a, b):
    return np.where(a * b > 0, np.where(np.abs(a) <= np.abs(b), a, b), 0.0)


def _idx(j, n, bc):
    return j % n if bc == 0 else min(max(j, 0), n - 1)


def step(cfg, f, lam):
    """cfg: dict with orbit table (4 or 6 orbits), gamma, S[nv], Q, omega1, omega2, T_ig,
    dx, dy, dt, bc_x, bc_y. f: [nv, ny, nx], lam: [ny, nx]."""
    vx, vy, eta = velocity_set(cfg["orbit_kind"], cfg["orbit_speed"], cfg["orbit_eta"])
    nv = len(vx)
    I = 2.0 / (cfg["gamma"] - 1.0) - D
    M = moment_matrix(vx, vy, eta)
    S = np.broadcast_to(np.asarray(cfg["S"], float), (nv,))
    ny, nx = lam.shape
    dx, dy, dt = cfg["dx"], cfg["dy"], cfg["dt"]
    bx, by = cfg["bc_x"], cfg["bc_y"]

    def at(a, x, y):  # field value with boundary condition applied
        return a[..., _idx(y, ny, by), _idx(x, nx, bx)]

    rho = f.sum(axis=0)
    ux = np.tensordot(vx, f, 1) / rho
    uy = np.tensordot(vy, f, 1) / rho
    E2 = np.tensordot(vx**2 + vy**2 + eta**2, f, 1)
    T = (E2 / rho - ux**2 - uy**2) / (D + I)

    f_new = np.empty_like(f)
    lam_new = np.empty_like(lam)
    for y in range(ny):
        for x in range(nx):
            r, u, v, t = rho[y, x], ux[y, x], uy[y, x], T[y, x]
            dux_dx = (at(ux, x + 1, y) - at(ux, x - 1, y)) / (2 * dx)
            duy_dx = (at(uy, x + 1, y) - at(uy, x - 1, y)) / (2 * dx)
            dux_dy = (at(ux, x, y + 1) - at(ux, x, y - 1)) / (2 * dy)
            duy_dy = (at(uy, x, y + 1) - at(uy, x, y - 1)) / (2 * dy)
            div = dux_dx + duy_dy
            fc = f[:, y, x]
            feq = np.linalg.solve(M, maxwellian_moments(r, u, v, t, I, nv=nv))
            coll = -np.linalg.solve(M, S * (M @ (fc - feq)))
            A = np.zeros(nv)
            A[7] = r * t * (S[4] - S[7]) / S[4] * (4 * u * (dux_dx - div / (D + I))
                                                   + 2 * v * (duy_dx + dux_dy))
            A[8] = r * t * (S[6] - S[8]) / S[6] * (4 * v * (duy_dy - div / (D + I))
                                                   + 2 * u * (duy_dx + dux_dy))
            l0 = lam[y, x]
            dl = 0.0
            if t > cfg["T_ig"]:
                a, b = cfg["omega1"] * r * t, cfg["omega2"] * r * t
                sol = solve_ivp(lambda _, z: (1 - z) * (a + b * z), (0, dt), [l0],
                                method="DOP853", rtol=1e-13, atol=1e-16)
                dl = sol.y[0, -1] - l0
            if nv == 16:
                Chat = (maxwellian_moments(r, u, v, t, I, dT=True) * 2 * cfg["Q"] * (dl / dt)
                        / (D + I))
                C = np.linalg.solve(M, Chat)
            else:
                shape = -(1 + D) * I * t + I * ((vx - u) ** 2 + (vy - v) ** 2) + eta**2
                C = feq * cfg["Q"] * shape / (I * (D + I) * t * t) * (dl / dt)
            Om = coll + np.linalg.solve(M, A) + C

            adv = np.zeros(nv)
            for i in range(nv):
                for vel, ax, h in ((vx[i], 0, dx), (vy[i], 1, dy)):
                    if vel == 0:
                        continue
                    g = [at(f[i], x + k * (ax == 0), y + k * (ax == 1)) for k in range(-2, 3)]
                    # g[0..4] = f_{j-2..j+2}
                    if vel > 0:
                        Hp = vel * (g[2] + 0.5 * _mm(g[2] - g[1], g[3] - g[2]))
                        Hm = vel * (g[1] + 0.5 * _mm(g[1] - g[0], g[2] - g[1]))
                    else:
                        Hp = vel * (g[3] - 0.5 * _mm(g[3] - g[2], g[4] - g[3]))
                        Hm = vel * (g[2] - 0.5 * _mm(g[2] - g[1], g[3] - g[2]))
                    adv[i] += (Hp - Hm) / h
            f_new[:, y, x] = fc + dt * (Om - adv)

            lg = 0.0
            for vel, ax, h in ((u, 0, dx), (v, 1, dy)):
                q = [at(lam, x + k * (ax == 0), y + k * (ax == 1)) for k in range(-2, 3)]
                if vel > 0:
                    right = q[2] + 0.5 * _mm(q[2] - q[1], q[3] - q[2])
                    left = q[1] + 0.5 * _mm(q[1] - q[0], q[2] - q[1])
                    lg += vel * (right - left) / h
                elif vel < 0:
                    right = q[3] - 0.5 * _mm(q[3] - q[2], q[4] - q[3])
                    left = q[2] - 0.5 * _mm(q[2] - q[1], q[3] - q[2])
                    lg += vel * (right - left) / h
            lam_new[y, x] = min(1.0, max(0.0, l0 - dt * lg + dl))
    return f_new, lam_new


def equilibrium(cfg, rho, ux, uy, T):
    vx, vy, eta = velocity_set(cfg["orbit_kind"], cfg["orbit_speed"], cfg["orbit_eta"])
    I = 2.0 / (cfg["gamma"] - 1.0) - D
    M = moment_matrix(vx, vy, eta)
    nv = len(vx)
    ny, nx = rho.shape
    f = np.empty((nv, ny, nx))
    for y in range(ny):
        for x in range(nx):
            f[:, y, x] = np.linalg.solve(M, maxwellian_moments(rho[y, x], ux[y, x], uy[y, x],
                                                               T[y, x], I, nv=nv))
    return f


def tne_record(cfg, f):
    """Grid-wide TNE record of a state, written from Sec. VI without the oracle: for every
    cell Delta_k = (M f)_k - f_hat^eq_k (k >= 5) with f_hat^eq from quadrature of the
    continuous Maxwellian at the cell's rho, u, T; Delta_1..4 vanish by conservation and are
    taken as 0. d = sqrt(sum_k Delta_k^2) (Eq. (91)). Sums of Delta_k, |Delta_k|, d and d^2
    are weighted by the cell area dx dy; min and max are per-cell values.
    Returns (delta [nv, ny, nx], dict like the oracle's record)."""
    vx, vy, eta = velocity_set(cfg["orbit_kind"], cfg["orbit_speed"], cfg["orbit_eta"])
    nv = len(vx)
    I = 2.0 / (cfg["gamma"] - 1.0) - D
    M = moment_matrix(vx, vy, eta)
    _, ny, nx = f.shape
    rho = f.sum(axis=0)
    ux = np.tensordot(vx, f, 1) / rho
    uy = np.tensordot(vy, f, 1) / rho
    T = (np.tensordot(vx**2 + vy**2 + eta**2, f, 1) / rho - ux**2 - uy**2) / (D + I)
    delta = np.zeros((nv, ny, nx))
    for y in range(ny):
        for x in range(nx):
            q = maxwellian_moments(rho[y, x], ux[y, x], uy[y, x], T[y, x], I, nv=nv)
            delta[4:, y, x] = (M @ f[:, y, x] - q)[4:]
    area = cfg["dx"] * cfg["dy"]
    d = np.sqrt((delta ** 2).sum(axis=0))
    rec = {"sum": delta.sum(axis=(1, 2)) * area, "abs_sum": np.abs(delta).sum(axis=(1, 2)) * area,
           "min": delta.min(axis=(1, 2)), "max": delta.max(axis=(1, 2)),
           "d_sum": float(d.sum() * area), "d2_sum": float((d ** 2).sum() * area)}
    return delta, rec
