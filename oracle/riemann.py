"""Exact solution of the one-dimensional Riemann problem of the ideal-gas
Euler equations: the analytic curves against which the paper checks its Sod
shock tube (Sec. 3, Sod shock tube test).  TEST INFRASTRUCTURE ONLY, like the
rest of ``oracle``.

A Riemann problem's solution is self-similar in xi = (x - x0)/t: a left wave
(shock or rarefaction), a contact moving with the star velocity u*, and a
right wave.  The star pressure p* is the root of

    F(p) = f_L(p) + f_R(p) + (u_R - u_L) = 0,

with, for K = L, R (c_K = sqrt(gamma p_K / rho_K)):

    shock (p > p_K):        f_K = (p - p_K) sqrt(A_K / (p + B_K)),
                            A_K = 2 / ((gamma + 1) rho_K),  B_K = p_K (gamma - 1)/(gamma + 1)
    rarefaction (p <= p_K): f_K = 2 c_K / (gamma - 1) ((p / p_K)^((gamma - 1)/(2 gamma)) - 1)

(the shock branch is the Rankine-Hugoniot jump, the rarefaction branch the
isentropic fan with its Riemann invariant); u* = (u_L + u_R)/2 + (f_R - f_L)/2.
This is the standard construction (e.g. E. F. Toro, Riemann Solvers and
Numerical Methods for Fluid Dynamics, Ch. 4), written from those relations.
F is monotone and concave in p, so Newton from below converges; a bisection
bracket guards it.
"""
from __future__ import annotations

import math

import numpy as np


def _f(p, rho, pk, gamma):
    """f_K(p) and its derivative for one side."""
    c = math.sqrt(gamma * pk / rho)
    if p > pk:
        A = 2.0 / ((gamma + 1.0) * rho)
        B = pk * (gamma - 1.0) / (gamma + 1.0)
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    e = (gamma - 1.0) / (2.0 * gamma)
    return 2.0 * c / (gamma - 1.0) * ((p / pk) ** e - 1.0), (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma)) / (rho * c)


def star_state(left, right, gamma):
    """(p*, u*) of the Riemann problem with states (rho, u, p) left and right.
    Raises if the states generate a vacuum (no positive p*)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(gamma * pl / rl), math.sqrt(gamma * pr / rr)
    du = ur - ul
    if 2.0 * (cl + cr) / (gamma - 1.0) <= du:
        raise ValueError("vacuum: the states separate")

    def F(p):
        a, da = _f(p, rl, pl, gamma)
        b, db = _f(p, rr, pr, gamma)
        return a + b + du, da + db

    lo, hi = 0.0, max(pl, pr)
    while F(hi)[0] < 0.0:
        hi *= 2.0
    p = 0.5 * (pl + pr)
    for _ in range(200):
        v, dv = F(p)
        if v > 0.0:
            hi = p
        else:
            lo = p
        pn = p - v / dv
        if not (lo < pn < hi):
            pn = 0.5 * (lo + hi)
        if abs(pn - p) <= 1e-16 * p:
            p = pn
            break
        p = pn
    fl = _f(p, rl, pl, gamma)[0]
    fr = _f(p, rr, pr, gamma)[0]
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(left, right, gamma, xi):
    """(rho, u, p) of the self-similar solution at xi = (x - x0)/t (array)."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, gamma)
    xi = np.asarray(xi, dtype=np.float64)
    rho, u, p = np.empty_like(xi), np.empty_like(xi), np.empty_like(xi)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    for k, s in np.ndenumerate(xi):
        if s <= us:                                   # left of the contact
            r0, u0, p0, sgn = rl, ul, pl, -1.0
        else:
            r0, u0, p0, sgn = rr, ur, pr, 1.0
        c0 = math.sqrt(gamma * p0 / r0)
        if ps > p0:                                   # shock
            S = u0 + sgn * c0 * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / p0 + (gamma - 1.0) / (2.0 * gamma))
            if sgn * (s - S) >= 0.0:                  # ahead of the shock
                rho[k], u[k], p[k] = r0, u0, p0
            else:
                rho[k] = r0 * (ps / p0 + g1) / (g1 * ps / p0 + 1.0)
                u[k], p[k] = us, ps
        else:                                         # rarefaction
            cs = c0 * (ps / p0) ** ((gamma - 1.0) / (2.0 * gamma))
            head, tail = u0 + sgn * c0, us + sgn * cs
            if sgn * (s - head) >= 0.0:
                rho[k], u[k], p[k] = r0, u0, p0
            elif sgn * (s - tail) <= 0.0:
                rho[k] = r0 * (ps / p0) ** (1.0 / gamma)
                u[k], p[k] = us, ps
            else:                                     # inside the fan: s = u + sgn c
                c = 2.0 / (gamma + 1.0) * (c0 - sgn * (gamma - 1.0) / 2.0 * (u0 - s))
                uu = s - sgn * c
                rho[k] = r0 * (c / c0) ** (2.0 / (gamma - 1.0))
                u[k], p[k] = uu, p0 * (c / c0) ** (2.0 * gamma / (gamma - 1.0))
    return rho, u, p


def shock_speed(left, right, gamma):
    """Speed of the right-moving shock when the right wave is a shock."""
    ps, _ = star_state(left, right, gamma)
    rr, ur, pr = right
    cr = math.sqrt(gamma * pr / rr)
    return ur + cr * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pr + (gamma - 1.0) / (2.0 * gamma))
