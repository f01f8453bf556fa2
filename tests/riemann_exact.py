"""Exact solution of the 1D Riemann problem for the Euler equations (ideal gas).

Test helper, independent of the scheme under test. The method is the standard one:
the star-region pressure solves f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is the
Rankine-Hugoniot shock relation for p > p_K and the isentropic rarefaction relation
for p <= p_K; Newton iteration from the two-rarefaction estimate; then the
self-similar solution is sampled at x/t (E. F. Toro, "Riemann Solvers and Numerical
Methods for Fluid Dynamics", 3rd ed., Springer 2009, Ch. 4).
"""
import math

import numpy as np


def _fK(p, rho, pK, c, g):
    if p > pK:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pK
        s = math.sqrt(A / (p + B))
        return (p - pK) * s, s * (1.0 - 0.5 * (p - pK) / (p + B))
    r = p / pK
    return 2.0 * c / (g - 1.0) * (r ** ((g - 1.0) / (2.0 * g)) - 1.0), r ** (-(g + 1.0) / (2.0 * g)) / (rho * c)


def star_state(left, right, g=1.4, tol=1e-14):
    """left/right = (rho, u, p). Returns (p_star, u_star)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    du = ur - ul
    z = (g - 1.0) / (2.0 * g)
    p = ((cl + cr - 0.5 * (g - 1.0) * du) / (cl / pl ** z + cr / pr ** z)) ** (1.0 / z)
    p = max(p, 1e-12)
    for _ in range(200):
        fl, dfl = _fK(p, rl, pl, cl, g)
        fr, dfr = _fK(p, rr, pr, cr, g)
        pn = p - (fl + fr + du) / (dfl + dfr)
        pn = max(pn, 1e-14 * p)
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fK(p, rl, pl, cl, g)
    fr, _ = _fK(p, rr, pr, cr, g)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(left, right, xi, g=1.4):
    """Density, velocity, pressure at similarity coordinates xi = (x - x0)/t (array)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    ps, us = star_state(left, right, g)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    gm = (g - 1.0) / (g + 1.0)
    for k, s in np.ndenumerate(xi):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                S = ul - cl * math.sqrt((g + 1.0) / (2 * g) * ps / pl + (g - 1.0) / (2 * g))
                if s <= S:
                    rho[k], u[k], p[k] = rl, ul, pl
                else:
                    rho[k], u[k], p[k] = rl * (ps / pl + gm) / (gm * ps / pl + 1.0), us, ps
            else:  # left rarefaction
                cs = cl * (ps / pl) ** ((g - 1.0) / (2 * g))
                if s <= ul - cl:
                    rho[k], u[k], p[k] = rl, ul, pl
                elif s >= us - cs:
                    rho[k], u[k], p[k] = rl * (ps / pl) ** (1.0 / g), us, ps
                else:
                    uu = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + s)
                    cc = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - s))
                    rho[k] = rl * (cc / cl) ** (2.0 / (g - 1.0))
                    u[k] = uu
                    p[k] = pl * (cc / cl) ** (2.0 * g / (g - 1.0))
        else:  # right of the contact
            if ps > pr:
                S = ur + cr * math.sqrt((g + 1.0) / (2 * g) * ps / pr + (g - 1.0) / (2 * g))
                if s >= S:
                    rho[k], u[k], p[k] = rr, ur, pr
                else:
                    rho[k], u[k], p[k] = rr * (ps / pr + gm) / (gm * ps / pr + 1.0), us, ps
            else:
                cs = cr * (ps / pr) ** ((g - 1.0) / (2 * g))
                if s >= ur + cr:
                    rho[k], u[k], p[k] = rr, ur, pr
                elif s <= us + cs:
                    rho[k], u[k], p[k] = rr * (ps / pr) ** (1.0 / g), us, ps
                else:
                    uu = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + s)
                    cc = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - s))
                    rho[k] = rr * (cc / cr) ** (2.0 / (g - 1.0))
                    u[k] = uu
                    p[k] = pr * (cc / cr) ** (2.0 * g / (g - 1.0))
    return rho, u, p
