"""Exact solution of the Riemann problem of the 1-D Euler equations for an ideal gas.

Test infrastructure: the reference profile for the shock-tube pins (the paper
compares its Sod, Lax and Sjogreen runs with exact Euler solutions, Sec. IV.B).
Written from the gas-dynamics relations: the star pressure solves
f_L(p) + f_R(p) + u_R - u_L = 0 with f_K the shock (Rankine-Hugoniot) or
rarefaction (isentropic) branch, then the self-similar solution is sampled at
x/t.
"""
from __future__ import annotations

import math

import numpy as np


def _f_branch(p, rho, pk, g):
    c = math.sqrt(g * pk / rho)
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(A / (p + B))
        f = (p - pk) * s
        df = s * (1.0 - 0.5 * (p - pk) / (p + B))
    else:  # rarefaction
        e = (g - 1.0) / (2.0 * g)
        f = 2.0 * c / (g - 1.0) * ((p / pk) ** e - 1.0)
        df = 1.0 / (rho * c) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(L, R, g):
    """(p*, u*) for left/right states (rho, u, p)."""
    rl, ul, pl = L
    rr, ur, pr = R
    p = max(1e-10, 0.5 * (pl + pr))
    for _ in range(200):
        fl, dl = _f_branch(p, rl, pl, g)
        fr, dr = _f_branch(p, rr, pr, g)
        F = fl + fr + ur - ul
        dp = F / (dl + dr)
        pn = max(1e-12, p - dp)
        if abs(pn - p) <= 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f_branch(p, rl, pl, g)
    fr, _ = _f_branch(p, rr, pr, g)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(L, R, g, xi):
    """(rho, u, p) at similarity coordinates xi = (x - x0) / t (array)."""
    rl, ul, pl = L
    rr, ur, pr = R
    ps, us = star_state(L, R, g)
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    xi = np.asarray(xi, float)
    rho, u, p = np.empty_like(xi), np.empty_like(xi), np.empty_like(xi)
    gm = (g - 1.0) / (g + 1.0)
    for n, s in enumerate(xi.flat):
        if s <= us:  # left of contact
            if ps > pl:  # left shock
                rs = rl * (ps / pl + gm) / (gm * ps / pl + 1.0)
                sl = ul - cl * math.sqrt((g + 1.0) / (2 * g) * ps / pl + (g - 1.0) / (2 * g))
                st = (rl, ul, pl) if s < sl else (rs, us, ps)
            else:  # left rarefaction
                rs = rl * (ps / pl) ** (1.0 / g)
                cs = cl * (ps / pl) ** ((g - 1.0) / (2 * g))
                if s < ul - cl:
                    st = (rl, ul, pl)
                elif s > us - cs:
                    st = (rs, us, ps)
                else:
                    uu = 2.0 / (g + 1.0) * (cl + (g - 1.0) / 2.0 * ul + s)
                    c = 2.0 / (g + 1.0) * (cl + (g - 1.0) / 2.0 * (ul - s))
                    rr_ = rl * (c / cl) ** (2.0 / (g - 1.0))
                    st = (rr_, uu, pl * (c / cl) ** (2.0 * g / (g - 1.0)))
        else:  # right of contact
            if ps > pr:  # right shock
                rs = rr * (ps / pr + gm) / (gm * ps / pr + 1.0)
                sr = ur + cr * math.sqrt((g + 1.0) / (2 * g) * ps / pr + (g - 1.0) / (2 * g))
                st = (rr, ur, pr) if s > sr else (rs, us, ps)
            else:  # right rarefaction
                rs = rr * (ps / pr) ** (1.0 / g)
                cs = cr * (ps / pr) ** ((g - 1.0) / (2 * g))
                if s > ur + cr:
                    st = (rr, ur, pr)
                elif s < us + cs:
                    st = (rs, us, ps)
                else:
                    uu = 2.0 / (g + 1.0) * (-cr + (g - 1.0) / 2.0 * ur + s)
                    c = 2.0 / (g + 1.0) * (cr - (g - 1.0) / 2.0 * (ur - s))
                    rr_ = rr * (c / cr) ** (2.0 / (g - 1.0))
                    st = (rr_, uu, pr * (c / cr) ** (2.0 * g / (g - 1.0)))
        rho.flat[n], u.flat[n], p.flat[n] = st
    return rho, u, p
