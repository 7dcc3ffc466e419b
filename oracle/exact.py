"""Closed-form reference solutions for the oracle's physics pins (test infrastructure).

* ``riemann_exact``: the exact solution of the 1-D Riemann problem for an ideal
  gas, written from the textbook construction (pressure function f_L + f_R +
  du = 0 solved by Newton's method, then self-similar sampling of shocks and
  rarefactions).  Used for the Sod tube of Sec. 5.1.2.
* ``l1_error``: the volume-weighted L1 norm of Sec. 5.1.1.

The isentropic vortex of Sec. 5.2.1 is an exact travelling solution; its
closed form is ``paper_1705_02028_gb300.inputs.vortex_primitives`` (the same
formula builds the initial state and, translated, the solution at time t).
"""
from __future__ import annotations

import math

import numpy as np


def _f_side(p, rho, pk, gamma):
    """Pressure function of one side and its derivative (shock for p > pk, else rarefaction)."""
    c = math.sqrt(gamma * pk / rho)
    if p > pk:
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    e = (gamma - 1.0) / (2.0 * gamma)
    r = (p / pk) ** e
    return 2.0 * c / (gamma - 1.0) * (r - 1.0), 1.0 / (rho * c) * (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma))


def star_state(left, right, gamma=1.4, tol=1e-14):
    """(p*, u*) of the Riemann problem left=(rho,u,p), right=(rho,u,p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    p = max(0.5 * (pl + pr), 1e-12)
    for _ in range(100):
        fl, dl = _f_side(p, rl, pl, gamma)
        fr, dr = _f_side(p, rr, pr, gamma)
        f = fl + fr + (ur - ul)
        pn = p - f / (dl + dr)
        if pn <= 0:
            pn = 0.5 * p
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f_side(p, rl, pl, gamma)
    fr, _ = _f_side(p, rr, pr, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def riemann_exact(left, right, xi, gamma=1.4):
    """Sample the exact solution at similarity coordinates xi = (x - x0) / t.

    Returns (rho, u, p) arrays."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, gamma)
    g = gamma
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    gm = (g - 1.0) / (g + 1.0)
    for n, s in np.ndenumerate(xi):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                sl = ul - cl * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if s <= sl:
                    rho[n], u[n], p[n] = rl, ul, pl
                else:
                    rho[n] = rl * (ps / pl + gm) / (gm * ps / pl + 1.0)
                    u[n], p[n] = us, ps
            else:  # left rarefaction
                cls = cl * (ps / pl) ** ((g - 1) / (2 * g))
                head, tail = ul - cl, us - cls
                if s <= head:
                    rho[n], u[n], p[n] = rl, ul, pl
                elif s >= tail:
                    rho[n] = rl * (ps / pl) ** (1.0 / g)
                    u[n], p[n] = us, ps
                else:
                    c = 2.0 / (g + 1) * (cl + (g - 1) / 2.0 * (ul - s))
                    u[n] = 2.0 / (g + 1) * (cl + (g - 1) / 2.0 * ul + s)
                    rho[n] = rl * (c / cl) ** (2.0 / (g - 1))
                    p[n] = pl * (c / cl) ** (2.0 * g / (g - 1))
        else:  # right of the contact
            if ps > pr:  # right shock
                sr = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if s >= sr:
                    rho[n], u[n], p[n] = rr, ur, pr
                else:
                    rho[n] = rr * (ps / pr + gm) / (gm * ps / pr + 1.0)
                    u[n], p[n] = us, ps
            else:  # right rarefaction
                crs = cr * (ps / pr) ** ((g - 1) / (2 * g))
                head, tail = ur + cr, us + crs
                if s >= head:
                    rho[n], u[n], p[n] = rr, ur, pr
                elif s <= tail:
                    rho[n] = rr * (ps / pr) ** (1.0 / g)
                    u[n], p[n] = us, ps
                else:
                    c = 2.0 / (g + 1) * (cr - (g - 1) / 2.0 * (ur - s))
                    u[n] = 2.0 / (g + 1) * (-cr + (g - 1) / 2.0 * ur + s)
                    rho[n] = rr * (c / cr) ** (2.0 / (g - 1))
                    p[n] = pr * (c / cr) ** (2.0 * g / (g - 1))
    return rho, u, p


def l1_error(V, a, b):
    """L1 = sum_i A_i |a_i - b_i| / sum_i A_i   (Sec. 5.1.1)."""
    V = np.asarray(V, dtype=np.float64)
    return float(np.sum(V * np.abs(np.asarray(a) - np.asarray(b))) / np.sum(V))
