"""Differentiable FP64 reference of the 1-D MRT-LBKM step in plain PyTorch (CPU).

TEST INFRASTRUCTURE ONLY (like the C oracle): the tests use it to obtain the exact
gradient of the discrete forward map by reverse-mode automatic differentiation,
against which the hand-written CUDA adjoint is checked. It implements the same
step as ``lbkm_oracle.c`` (Sec. II of the paper, CE sign of A_hat per Eq. (29),
chemical term in moment space per Eqs. (19)-(23), reaction Eq. (28) integrated
exactly over dt, NND advection, forward Euler) for Ny = 1 with zero-gradient (or periodic)
ghost cells, written independently with whole-array operations.

Non-smooth points take the conventions the adjoint uses: the ignition test
T > T_ig is a hard switch (no derivative through it), minmod follows the branch
that the values select, and the clamp of lambda to [0, 1] passes the derivative
when the unclamped value lies inside or on the bounds.
"""
from __future__ import annotations

import numpy as np
import torch

D = 2.0


def _moment_rows(vx, vy, eta):
    w = vx * vx + vy * vy + eta * eta
    return torch.stack([torch.ones_like(vx), vx, vy, w, vx * vx, vx * vy, vy * vy, w * vx,
                        w * vy, vx ** 3, vx * vx * vy, vx * vy * vy, vy ** 3, w * vx * vx,
                        w * vx * vy, w * vy * vy])


def _velocities(orbit_kind, orbit_speed, orbit_eta):
    axis = [(1, 0), (0, 1), (-1, 0), (0, -1)]
    diag = [(1, 1), (-1, 1), (-1, -1), (1, -1)]
    vx, vy, eta = [], [], []
    for kind, c, e in zip(orbit_kind, orbit_speed, orbit_eta):
        for a, b in (axis if kind == 0 else diag):
            vx.append(c * a)
            vy.append(c * b)
            eta.append(e)
    t = lambda a: torch.tensor(a, dtype=torch.float64)
    return t(vx), t(vy), t(eta)


def _feq(rho, ux, uy, T, DI):
    """f_hat^eq_1..16 (list after Eq. (16), entries 14 and 16 per Eq. (11)); [16, n]."""
    u2 = ux * ux + uy * uy
    A = (DI + 2) * T + u2
    B = (DI + 4) * T + u2
    return torch.stack([rho, rho * ux, rho * uy, rho * (DI * T + u2), rho * (T + ux * ux),
                        rho * ux * uy, rho * (T + uy * uy), rho * ux * A, rho * uy * A,
                        3 * rho * ux * T + rho * ux ** 3, rho * uy * T + rho * ux * ux * uy,
                        rho * ux * T + rho * ux * uy * uy, 3 * rho * uy * T + rho * uy ** 3,
                        rho * A * T + rho * ux * ux * B, rho * ux * uy * B,
                        rho * A * T + rho * uy * uy * B])


def _dfeq_dT(rho, ux, uy, T, DI):
    u2 = ux * ux + uy * uy
    dAT = 2 * (DI + 2) * T + u2
    z = torch.zeros_like(rho)
    return torch.stack([z, z, z, rho * DI, rho, z, rho, rho * ux * (DI + 2), rho * uy * (DI + 2),
                        3 * rho * ux, rho * uy, rho * ux, 3 * rho * uy,
                        rho * dAT + rho * ux * ux * (DI + 4), rho * ux * uy * (DI + 4),
                        rho * dAT + rho * uy * uy * (DI + 4)])


_RECORD = None  # list collecting branch patterns when set (finite-difference checks)


def _note(mask):
    if _RECORD is not None:
        _RECORD.append(mask.detach().clone())


def _mm(a, b):
    same = a * b > 0
    first = a.abs() <= b.abs()
    if _RECORD is not None:  # branches that change the value by more than rounding
        big = (a.abs() > 1e-13) & (b.abs() > 1e-13)
        _note(same & big)
        _note(first & big & ((a.abs() - b.abs()).abs() > 1e-13))
    return torch.where(same, torch.where(first, a, b), torch.zeros_like(a))


def record_branches(fn):
    """Run fn() and return (its result, a list of every branch mask it took)."""
    global _RECORD
    _RECORD = []
    try:
        out = fn()
        return out, _RECORD
    finally:
        _RECORD = None


def _pad(a, periodic=False):
    """Two ghost cells on each side along the last axis: zero-gradient copies of the end
    cells, or the periodic images."""
    if periodic:
        return torch.cat([a[..., -2:], a, a[..., :2]], dim=-1)
    return torch.cat([a[..., :1], a[..., :1], a, a[..., -1:], a[..., -1:]], dim=-1)


class Model1D:
    """Set-up shared by the forward map and its objective."""

    def __init__(self, nx, *, gamma, orbit_kind, orbit_speed, orbit_eta, T_ig, dx, dt,
                 omega2=0.0, periodic=False):
        self.nx = nx
        self.vx, self.vy, self.eta = _velocities(orbit_kind, orbit_speed, orbit_eta)
        self.M = _moment_rows(self.vx, self.vy, self.eta)
        self.Minv = torch.linalg.inv(self.M)
        self.I = 2.0 / (gamma - 1.0) - D
        self.DI = D + self.I
        self.T_ig, self.dx, self.dt, self.omega2 = T_ig, dx, dt, omega2
        self.periodic = periodic

    def init(self, rho, ux, uy, T):
        return self.Minv @ _feq(rho, ux, uy, T, self.DI)

    def macros(self, f):
        m = self.M @ f
        rho = m[0]
        ux, uy = m[1] / rho, m[2] / rho
        T = (m[3] / rho - ux * ux - uy * uy) / self.DI
        return m, rho, ux, uy, T

    def delta(self, f):
        m, rho, ux, uy, T = self.macros(f)
        return m[4:] - _feq(rho, ux, uy, T, self.DI)[4:]

    def step(self, f, lam, S, Q, omega1):
        """(f, lambda) at t_n -> t_n+1; S: [16], Q, omega1: scalars (tensors)."""
        dt, dx, DI = self.dt, self.dx, self.DI
        m, rho, ux, uy, T = self.macros(f)
        q = _feq(rho, ux, uy, T, DI)
        Dk = m[4:] - q[4:]
        uxp, uyp = _pad(ux, self.periodic), _pad(uy, self.periodic)
        gx = (uxp[3:-1] - uxp[1:-3]) / (2 * dx)
        gy = (uyp[3:-1] - uyp[1:-3]) / (2 * dx)
        th = gx / DI
        A8 = rho * T * (S[4] - S[7]) / S[4] * (4 * ux * (gx - th) + 2 * uy * gy)
        A9 = rho * T * (S[6] - S[8]) / S[6] * (4 * uy * (-th) + 2 * ux * gy)
        lam0 = lam
        p = rho * T
        a = omega1 * p
        b = self.omega2 * p
        mu0 = 1 - lam0
        if self.omega2 == 0.0:
            mu = mu0 * torch.exp(-a * dt)
        else:
            k = a + b
            e = torch.exp(-k * dt)
            mu = k * mu0 * e / (k - b * mu0 * (1 - e))
        _note(T > self.T_ig)
        dl = torch.where(T > self.T_ig, mu0 - mu, torch.zeros_like(T))
        cr = dl * 2 * Q / (DI * dt)
        dq = _dfeq_dT(rho, ux, uy, T, DI)
        om_hat = torch.cat([torch.zeros(3, self.nx, dtype=f.dtype), (dq[3] * cr)[None],
                            -S[4:, None] * Dk + dq[4:] * cr[None]])
        om_hat = om_hat + torch.stack([torch.zeros_like(A8)] * 7 + [A8, A9] +
                                      [torch.zeros_like(A8)] * 7)
        Om = self.Minv @ om_hat
        fp = _pad(f, self.periodic)
        adv = []
        for i in range(16):
            v = float(self.vx[i])
            g = [fp[i, k:k + self.nx] for k in range(5)]  # f_{j-2..j+2}
            if v > 0:
                Hp = g[2] + 0.5 * _mm(g[2] - g[1], g[3] - g[2])
                Hm = g[1] + 0.5 * _mm(g[1] - g[0], g[2] - g[1])
                adv.append(v * (Hp - Hm) / dx)
            elif v < 0:
                Hp = g[3] - 0.5 * _mm(g[3] - g[2], g[4] - g[3])
                Hm = g[2] - 0.5 * _mm(g[2] - g[1], g[3] - g[2])
                adv.append(v * (Hp - Hm) / dx)
            else:
                adv.append(torch.zeros(self.nx, dtype=f.dtype))
        f_new = f + dt * (Om - torch.stack(adv))
        lp = _pad(lam0, self.periodic)
        g = [lp[k:k + self.nx] for k in range(5)]
        Lp = (g[2] + 0.5 * _mm(g[2] - g[1], g[3] - g[2])) - (g[1] + 0.5 * _mm(g[1] - g[0], g[2] - g[1]))
        Ln = (g[3] - 0.5 * _mm(g[3] - g[2], g[4] - g[3])) - (g[2] - 0.5 * _mm(g[2] - g[1], g[3] - g[2]))
        ladv = torch.where(ux > 0, ux * Lp, torch.where(ux < 0, ux * Ln, torch.zeros_like(ux))) / dx
        raw = lam0 - dt * ladv + dl
        _note(ux > 0)
        _note(ux < 0)
        _note(raw < 0)
        _note(raw > 1)
        lam_new = torch.clamp(raw, 0.0, 1.0)
        return f_new, lam_new, Dk


def objective(model, rho0, ux0, uy0, T0, lam0, S, Q, omega1, steps, rho_target, w_tne,
              checkpoint_every=0, restarts=None):
    """J = 1/2 sum_x (rho_N - rho*)^2 dx + w_tne sum_{n<N} sum_x d_n^2 dx dt, d_n^2 = sum_k
    Delta_k^2 of the state entering step n. Returns (J, mismatch part, TNE part).
    omega2 of the model may be a tensor that requires a gradient.

    restarts: (f, lambda) for the steps 0, C, 2C, ... (C = checkpoint_every): each
    segment of C steps starts from the given state instead of the one the previous
    segment reached, the derivative passing to the reached state unchanged -- the
    objective and gradient of FP64 segments restarted from another run's states."""

    f = model.init(rho0, ux0, uy0, T0)
    lam = lam0
    tne = torch.zeros((), dtype=torch.float64)
    if restarts is not None and not checkpoint_every:
        raise ValueError("restarts need checkpoint_every")

    def seg(f, lam, S, Q, omega1, n):
        t = torch.zeros((), dtype=torch.float64)
        for _ in range(n):
            f, lam, Dk = model.step(f, lam, S, Q, omega1)
            t = t + (Dk * Dk).sum() * model.dx * model.dt
        return f, lam, t

    done = 0
    while done < steps:
        if restarts is not None:
            rf, rl = restarts[done // checkpoint_every]
            f = f + (torch.as_tensor(rf, dtype=torch.float64) - f).detach()
            lam = lam + (torch.as_tensor(rl, dtype=torch.float64) - lam).detach()
        n = min(checkpoint_every or steps, steps - done)
        if checkpoint_every:
            from torch.utils.checkpoint import checkpoint
            f, lam, t = checkpoint(seg, f, lam, S, Q, omega1, n, use_reentrant=False)
        else:
            f, lam, t = seg(f, lam, S, Q, omega1, n)
        tne = tne + t
        done += n
    rho = (model.M[0] @ f)
    mis = 0.5 * ((rho - rho_target) ** 2).sum() * model.dx
    return mis + w_tne * tne, mis, tne


def to_t(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float64))
