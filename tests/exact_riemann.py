"""Exact solution of the 1D Euler Riemann problem for an ideal gas.

Textbook method (E. F. Toro, "Riemann Solvers and Numerical Methods for Fluid
Dynamics", Ch. 4): Newton iteration on the star pressure using the shock /
rarefaction wave curves, then sampling of the self-similar solution.  Used only
as an independent reference for the oracle's Sod test.
"""
import math

import numpy as np


def _wave_curve(p, rho, pk, ck, gamma):
    if p > pk:  # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        q = math.sqrt(A / (p + B))
        f = (p - pk) * q
        df = q * (1.0 - 0.5 * (p - pk) / (B + p))
    else:       # rarefaction
        e = (gamma - 1.0) / (2.0 * gamma)
        f = 2.0 * ck / (gamma - 1.0) * ((p / pk) ** e - 1.0)
        df = 1.0 / (rho * ck) * (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma))
    return f, df


def star_state(rl, ul, pl, rr, ur, pr, gamma):
    cl = math.sqrt(gamma * pl / rl)
    cr = math.sqrt(gamma * pr / rr)
    p = max(1e-12, 0.5 * (pl + pr))
    for _ in range(100):
        fl, dfl = _wave_curve(p, rl, pl, cl, gamma)
        fr, dfr = _wave_curve(p, rr, pr, cr, gamma)
        dp = (fl + fr + ur - ul) / (dfl + dfr)
        p_new = max(1e-14, p - dp)
        if abs(p_new - p) < 1e-15 * (p_new + p):
            p = p_new
            break
        p = p_new
    fl, _ = _wave_curve(p, rl, pl, cl, gamma)
    fr, _ = _wave_curve(p, rr, pr, cr, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    g = gamma
    if p > pl:
        rsl = rl * ((p / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pl + 1))
    else:
        rsl = rl * (p / pl) ** (1 / g)
    if p > pr:
        rsr = rr * ((p / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pr + 1))
    else:
        rsr = rr * (p / pr) ** (1 / g)
    return p, u, rsl, rsr


def sample(x, t, x0, left, right, gamma):
    """Density, velocity, pressure at positions x (array) and time t."""
    rl, ul, pl = left
    rr, ur, pr = right
    g = gamma
    ps, us, rsl, rsr = star_state(rl, ul, pl, rr, ur, pr, g)
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    out = np.zeros((3, len(x)))
    for n, xx in enumerate(x):
        s = (xx - x0) / t
        if s <= us:  # left of contact
            if ps > pl:
                sl = ul - cl * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                out[:, n] = (rl, ul, pl) if s <= sl else (rsl, us, ps)
            else:
                shl = ul - cl
                csl = cl * (ps / pl) ** ((g - 1) / (2 * g))
                stl = us - csl
                if s <= shl:
                    out[:, n] = (rl, ul, pl)
                elif s >= stl:
                    out[:, n] = (rsl, us, ps)
                else:
                    c = 2 / (g + 1) * (cl + (g - 1) / 2 * (ul - s))
                    u = 2 / (g + 1) * (cl + (g - 1) / 2 * ul + s)
                    rho = rl * (c / cl) ** (2 / (g - 1))
                    out[:, n] = (rho, u, pl * (c / cl) ** (2 * g / (g - 1)))
        else:
            if ps > pr:
                sr = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                out[:, n] = (rr, ur, pr) if s >= sr else (rsr, us, ps)
            else:
                shr = ur + cr
                csr = cr * (ps / pr) ** ((g - 1) / (2 * g))
                str_ = us + csr
                if s >= shr:
                    out[:, n] = (rr, ur, pr)
                elif s <= str_:
                    out[:, n] = (rsr, us, ps)
                else:
                    c = 2 / (g + 1) * (cr - (g - 1) / 2 * (ur - s))
                    u = 2 / (g + 1) * (-cr + (g - 1) / 2 * ur + s)
                    rho = rr * (c / cr) ** (2 / (g - 1))
                    out[:, n] = (rho, u, pr * (c / cr) ** (2 * g / (g - 1)))
    return out
