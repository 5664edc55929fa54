"""Exact solution of the 1D Euler Riemann problem for an ideal gas.

Used only as a pin for the oracle (the Sod tube).  Written from the standard
derivation: the star-region pressure p* is the root of
    f(p) = f_L(p) + f_R(p) + (u_R - u_L) = 0,
with f_K the shock (p > p_K, Rankine-Hugoniot) or rarefaction (p <= p_K,
isentropic) relation of side K, solved here by bracketing and bisection/Brent.
The solution is then sampled along x/t.
"""
from __future__ import annotations

import math

import numpy as np


def _fK(p, rho, pK, gamma):
    c = math.sqrt(gamma * pK / rho)
    if p > pK:
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pK
        return (p - pK) * math.sqrt(A / (p + B))
    return 2.0 * c / (gamma - 1.0) * ((p / pK) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)


def star_state(left, right, gamma=1.4):
    rl, ul, pl = left
    rr, ur, pr = right

    def f(p):
        return _fK(p, rl, pl, gamma) + _fK(p, rr, pr, gamma) + (ur - ul)

    lo, hi = 1e-14, max(pl, pr)
    while f(hi) < 0.0:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0.0:
            hi = mid
        else:
            lo = mid
    ps = 0.5 * (lo + hi)
    us = 0.5 * (ul + ur) + 0.5 * (_fK(ps, rr, pr, gamma) - _fK(ps, rl, pl, gamma))
    return ps, us


def sample(left, right, xi, gamma=1.4):
    """Primitive (rho, u, p) at similarity coordinates xi = (x - x0)/t."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, gamma)
    cl = math.sqrt(gamma * pl / rl)
    cr = math.sqrt(gamma * pr / rr)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    out = np.zeros((3, len(xi)))
    for k, s in enumerate(np.asarray(xi, dtype=float)):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                SL = ul - cl * math.sqrt((gamma + 1) / (2 * gamma) * ps / pl + (gamma - 1) / (2 * gamma))
                if s <= SL:
                    w = (rl, ul, pl)
                else:
                    w = (rl * (ps / pl + g1) / (g1 * ps / pl + 1.0), us, ps)
            else:  # left rarefaction
                csl = cl * (ps / pl) ** ((gamma - 1) / (2 * gamma))
                if s <= ul - cl:
                    w = (rl, ul, pl)
                elif s >= us - csl:
                    w = (rl * (ps / pl) ** (1.0 / gamma), us, ps)
                else:
                    u = 2.0 / (gamma + 1) * (cl + (gamma - 1) / 2 * ul + s)
                    c = 2.0 / (gamma + 1) * (cl + (gamma - 1) / 2 * (ul - s))
                    rho = rl * (c / cl) ** (2.0 / (gamma - 1))
                    w = (rho, u, pl * (c / cl) ** (2 * gamma / (gamma - 1)))
        else:  # right of the contact
            if ps > pr:  # right shock
                SR = ur + cr * math.sqrt((gamma + 1) / (2 * gamma) * ps / pr + (gamma - 1) / (2 * gamma))
                if s >= SR:
                    w = (rr, ur, pr)
                else:
                    w = (rr * (ps / pr + g1) / (g1 * ps / pr + 1.0), us, ps)
            else:  # right rarefaction
                csr = cr * (ps / pr) ** ((gamma - 1) / (2 * gamma))
                if s >= ur + cr:
                    w = (rr, ur, pr)
                elif s <= us + csr:
                    w = (rr * (ps / pr) ** (1.0 / gamma), us, ps)
                else:
                    u = 2.0 / (gamma + 1) * (-cr + (gamma - 1) / 2 * ur + s)
                    c = 2.0 / (gamma + 1) * (cr - (gamma - 1) / 2 * (ur - s))
                    rho = rr * (c / cr) ** (2.0 / (gamma - 1))
                    w = (rho, u, pr * (c / cr) ** (2 * gamma / (gamma - 1)))
        out[:, k] = w
    return out


def sod_density(x, t, x0=0.5, gamma=1.4):
    return sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), (np.asarray(x) - x0) / t, gamma)[0]
