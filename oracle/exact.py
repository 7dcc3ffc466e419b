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


# ---------------------------------------------------------------------------
# Strong blast wave: the similarity solution of App. B
# ---------------------------------------------------------------------------
def _sedov_rhs(eta, y, a, gamma):
    """d/d eta of (rho^, v^, P^) for the self-similar strong blast of App. B.

    The three conditions are the continuity and momentum equations in the
    similarity variable, as App. B writes them, and the adiabatic condition
    D/Dt ln(P rho^-gamma) = 0 (equivalent to App. B's energy equation for
    smooth flow), derived here from the ansatz rho = rho_2 rho^, v = c_v r/t v^,
    P = c_p rho_1 r^2/t^2 P^, eta = r (E t^2 / rho_1)^(-1/(3+a)),
    c_v = 4 / ((3+a)(gamma+1)).  Each is linear in the three derivatives, which
    are found by a 3x3 solve."""
    rho, v, P = y
    g1 = gamma + 1.0
    cv = 4.0 / ((3.0 + a) * g1)
    k = 2.0 * eta / (3.0 + a)
    M = np.array([
        # continuity: -eta rho' + 2/(g+1) (rho v + eta rho' v + eta rho v') + 2a/(g+1) rho v = 0
        [-eta + 2.0 * eta * v / g1, 2.0 * eta * rho / g1, 0.0],
        # momentum: -(3+a) v - 2 eta v' + 4/(g+1) v (v + eta v') + 2 (g-1)/(g+1) (2P + eta P') / rho = 0
        [0.0, -2.0 * eta + 4.0 * eta * v / g1, 2.0 * (gamma - 1.0) / g1 * eta / rho],
        # adiabatic: -2 - k P'/P + gamma k rho'/rho + cv v (2 + eta P'/P - gamma eta rho'/rho) = 0
        [gamma * (k - cv * v * eta) / rho, 0.0, (-k + cv * v * eta) / P],
    ])
    rhs = -np.array([
        2.0 * rho * v / g1 + 2.0 * a * rho * v / g1,
        -(3.0 + a) * v + 4.0 * v * v / g1 + 4.0 * (gamma - 1.0) / g1 * P / rho,
        -2.0 + 2.0 * cv * v,
    ])
    return np.linalg.solve(M, rhs)


def sedov_profile(a, gamma, n=4000, x_min=1e-4):
    """Post-shock profiles rho^, v^, P^ of App. B as functions of x = eta / eta_s in
    [x_min, 1] (they do not depend on eta_s: the equations contain eta only through
    eta d/d eta), integrated inwards from the strong-shock values 1, 1, 1 with a
    classical fourth-order Runge-Kutta scheme on a grid uniform in ln x."""
    s = np.linspace(0.0, math.log(x_min), n)        # s = ln x, from the shock inwards
    y = np.array([1.0, 1.0, 1.0])
    out = np.empty((n, 3))
    out[0] = y
    f = lambda s_, y_: math.exp(s_) * _sedov_rhs(math.exp(s_), y_, a, gamma)   # dy/ds = x dy/dx
    for i in range(n - 1):
        h = s[i + 1] - s[i]
        k1 = f(s[i], y)
        k2 = f(s[i] + h / 2, y + h / 2 * k1)
        k3 = f(s[i] + h / 2, y + h / 2 * k2)
        k4 = f(s[i] + h, y + h * k3)
        y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        out[i + 1] = y
    return np.exp(s), out


def sedov_eta_shock(a, gamma, b, n=4000):
    """Shock position eta_s of the strong blast from App. B's energy constraint
    8 b / ((3+a)^2 (gamma^2 - 1)) int_0^eta_s (rho^ v^2 + P^) eta^(2+a) d eta = 1;
    b = 4 pi (sphere), 2 pi (cylinder), 2 (plane symmetric about x = 0, both sides)."""
    x, y = sedov_profile(a, gamma, n)
    w = (y[:, 0] * y[:, 1] ** 2 + y[:, 2]) * x ** (2 + a)
    # trapezoid in x (the integrand vanishes at x = 0 faster than x^(2+a))
    I = float(np.sum(0.5 * (w[1:] + w[:-1]) * (x[:-1] - x[1:])))
    return ((3 + a) ** 2 * (gamma ** 2 - 1) / (8.0 * b * I)) ** (1.0 / (3 + a))


def sedov_solution(r, t, E, rho1, a, gamma, b, n=4000):
    """(rho, v, P) of the strong blast at distances r >= 0 from the explosion at time t
    (pre-shock gas at rest with density rho1 and zero pressure)."""
    eta_s = sedov_eta_shock(a, gamma, b, n)
    R = eta_s * (E * t * t / rho1) ** (1.0 / (3 + a))
    x, y = sedov_profile(a, gamma, n)
    r = np.asarray(r, dtype=np.float64)
    xi = r / R
    inside = xi < 1.0
    xs, ys = x[::-1], y[::-1]                        # ascending x for interpolation
    rho = np.full(r.shape, rho1)
    v = np.zeros(r.shape)
    P = np.zeros(r.shape)
    rho2 = (gamma + 1.0) / (gamma - 1.0) * rho1
    cv = 4.0 / ((3.0 + a) * (gamma + 1.0))
    cp = 8.0 / ((3.0 + a) ** 2 * (gamma + 1.0))
    xi_in = np.clip(xi[inside], xs[0], 1.0)
    rho[inside] = rho2 * np.interp(xi_in, xs, ys[:, 0])
    v[inside] = cv * r[inside] / t * np.interp(xi_in, xs, ys[:, 1])
    P[inside] = cp * rho1 * r[inside] ** 2 / t ** 2 * np.interp(xi_in, xs, ys[:, 2])
    return rho, v, P, R
