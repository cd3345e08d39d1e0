"""Exact solution of the 1D Riemann problem for the Euler equations (ideal gas).

Used only to pin the oracle: the first-order scheme of the paper (Sec. 6.2)
must converge toward this solution on a triangulated shock-tube strip.
Written from the classical closed form: the star pressure solves
f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is the shock (Rankine-Hugoniot)
branch for p > p_K and the rarefaction (isentropic) branch otherwise; the
solution is self-similar in x/t.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq


def _f_branch(p, rho, pk, ck, g):
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        return (p - pk) * math.sqrt(A / (p + B))
    return 2.0 * ck / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)


def star_state(left, right, g=1.4):
    """(p*, u*, rho*_L, rho*_R) for primitive states (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    fun = lambda p: _f_branch(p, rl, pl, cl, g) + _f_branch(p, rr, pr, cr, g) + (ur - ul)  # noqa
    p = brentq(fun, 1e-12, 100.0 * max(pl, pr), xtol=1e-15, rtol=1e-15, maxiter=500)
    u = 0.5 * (ul + ur) + 0.5 * (_f_branch(p, rr, pr, cr, g) - _f_branch(p, rl, pl, cl, g))
    gm = (g - 1.0) / (g + 1.0)

    def rho_star(rk, pk):
        if p > pk:
            return rk * (p / pk + gm) / (gm * p / pk + 1.0)
        return rk * (p / pk) ** (1.0 / g)

    return p, u, rho_star(rl, pl), rho_star(rr, pr)


def sample(left, right, xi, g=1.4):
    """Primitive (rho, u, p) at similarity coordinates xi = (x - x0)/t."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    ps, us, rsl, rsr = star_state(left, right, g)
    xi = np.atleast_1d(np.asarray(xi, np.float64))
    out = np.empty((xi.size, 3))
    for i, s in enumerate(xi):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                sl = ul - cl * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                out[i] = (rl, ul, pl) if s < sl else (rsl, us, ps)
            else:  # left rarefaction
                csl = cl * (ps / pl) ** ((g - 1) / (2 * g))
                head, tail = ul - cl, us - csl
                if s < head:
                    out[i] = (rl, ul, pl)
                elif s > tail:
                    out[i] = (rsl, us, ps)
                else:
                    u = 2.0 / (g + 1) * (cl + (g - 1) / 2 * ul + s)
                    c = 2.0 / (g + 1) * (cl + (g - 1) / 2 * (ul - s))
                    rho = rl * (c / cl) ** (2 / (g - 1))
                    out[i] = (rho, u, pl * (c / cl) ** (2 * g / (g - 1)))
        else:  # right of the contact
            if ps > pr:  # right shock
                sr = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                out[i] = (rr, ur, pr) if s > sr else (rsr, us, ps)
            else:  # right rarefaction
                csr = cr * (ps / pr) ** ((g - 1) / (2 * g))
                head, tail = ur + cr, us + csr
                if s > head:
                    out[i] = (rr, ur, pr)
                elif s < tail:
                    out[i] = (rsr, us, ps)
                else:
                    u = 2.0 / (g + 1) * (-cr + (g - 1) / 2 * ur + s)
                    c = 2.0 / (g + 1) * (cr - (g - 1) / 2 * (ur - s))
                    rho = rr * (c / cr) ** (2 / (g - 1))
                    out[i] = (rho, u, pr * (c / cr) ** (2 * g / (g - 1)))
    return out
