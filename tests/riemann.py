"""Exact solution of the 1D Riemann problem for an ideal gas (test helper).

The classical construction: the star pressure solves f_L(p) + f_R(p) + (u_R - u_L) = 0, with
shock or rarefaction branches on each side; the solution is self-similar in s = x / t.
Used only to pin the compressible models (tolerance, not parity).
"""
import numpy as np


def _f(p, rho, pk, ck, g):
    if p > pk:                               # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        return (p - pk) * np.sqrt(A / (p + B))
    return 2.0 * ck / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)


def star_pressure(L, R, g):
    rl, ul, pl = L
    rr, ur, pr = R
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    lo, hi = 1e-12, 10 * max(pl, pr)
    for _ in range(200):                     # bisection: monotone function of p
        mid = 0.5 * (lo + hi)
        val = _f(mid, rl, pl, cl, g) + _f(mid, rr, pr, cr, g) + ur - ul
        if val > 0:
            hi = mid
        else:
            lo = mid
    ps = 0.5 * (lo + hi)
    us = 0.5 * (ul + ur) + 0.5 * (_f(ps, rr, pr, cr, g) - _f(ps, rl, pl, cl, g))
    return ps, us


def sample(L, R, g, s):
    """(rho, u, p) at similarity coordinates s = (x - x0)/t (array)."""
    rl, ul, pl = L
    rr, ur, pr = R
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    ps, us = star_pressure(L, R, g)
    out = np.zeros((3, s.size))
    for k, x in enumerate(s):
        if x <= us:                          # left of contact
            if ps > pl:                      # left shock
                rs = rl * ((ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1))
                sl = ul - cl * np.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                out[:, k] = (rl, ul, pl) if x < sl else (rs, us, ps)
            else:                            # left rarefaction
                rs = rl * (ps / pl) ** (1 / g)
                cs = cl * (ps / pl) ** ((g - 1) / (2 * g))
                if x < ul - cl:
                    out[:, k] = (rl, ul, pl)
                elif x > us - cs:
                    out[:, k] = (rs, us, ps)
                else:
                    u = 2 / (g + 1) * (cl + (g - 1) / 2 * ul + x)
                    c = 2 / (g + 1) * (cl + (g - 1) / 2 * (ul - x))
                    rho = rl * (c / cl) ** (2 / (g - 1))
                    out[:, k] = (rho, u, pl * (c / cl) ** (2 * g / (g - 1)))
        else:
            if ps > pr:                      # right shock
                rs = rr * ((ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1))
                sr = ur + cr * np.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                out[:, k] = (rr, ur, pr) if x > sr else (rs, us, ps)
            else:
                rs = rr * (ps / pr) ** (1 / g)
                cs = cr * (ps / pr) ** ((g - 1) / (2 * g))
                if x > ur + cr:
                    out[:, k] = (rr, ur, pr)
                elif x < us + cs:
                    out[:, k] = (rs, us, ps)
                else:
                    u = 2 / (g + 1) * (-cr + (g - 1) / 2 * ur + x)
                    c = 2 / (g + 1) * (cr - (g - 1) / 2 * (ur - x))
                    rho = rr * (c / cr) ** (2 / (g - 1))
                    out[:, k] = (rho, u, pr * (c / cr) ** (2 * g / (g - 1)))
    return out
