"""Exact solution of the Riemann problem of the 1-D Euler equations for a polytropic ideal
gas (the textbook construction: the star-region pressure is the root of
f_L(p) + f_R(p) + u_R - u_L = 0, with f_K the shock (Rankine-Hugoniot) or rarefaction
(isentropic) branch, solved by Newton's method; the solution is then sampled in x / t).
Used to pin the shock-tube runs (Sec. VI B) of the oracle and of the GPU path; it holds
none of the lattice Boltzmann scheme's arithmetic.
"""
from __future__ import annotations

import numpy as np


def _f(p, rho, pk, gamma):
    """f_K(p) and its derivative for one side of state (rho, pk)."""
    c = np.sqrt(gamma * pk / rho)
    if p > pk:  # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        q = np.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (p + B))
    e = (gamma - 1.0) / (2.0 * gamma)  # rarefaction
    return 2.0 * c / (gamma - 1.0) * ((p / pk) ** e - 1.0), (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma)) / (rho * c)


def star_state(left, right, gamma):
    """(p*, u*) of left = (rho, u, p), right = (rho, u, p)."""
    (rl, ul, pl), (rr, ur, pr) = left, right
    p = 0.5 * (pl + pr)
    for _ in range(100):
        fl, dl = _f(p, rl, pl, gamma)
        fr, dr = _f(p, rr, pr, gamma)
        dp = (fl + fr + ur - ul) / (dl + dr)
        p = max(p - dp, 1e-12)
        if abs(dp) < 1e-14 * p:
            break
    fl, _ = _f(p, rl, pl, gamma)
    fr, _ = _f(p, rr, pr, gamma)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(s, left, right, gamma):
    """(rho, u, p) at the similarity coordinates s = x / t (array)."""
    (rl, ul, pl), (rr, ur, pr) = left, right
    ps, us = star_state(left, right, gamma)
    g1, g2 = (gamma - 1.0) / (gamma + 1.0), (gamma - 1.0) / (2.0 * gamma)
    out = np.zeros((3, len(s)))
    for j, x in enumerate(np.asarray(s, float)):
        if x <= us:  # left of the contact
            rho, u, pk, sgn = rl, ul, pl, -1.0
        else:
            rho, u, pk, sgn = rr, ur, pr, 1.0
        c = np.sqrt(gamma * pk / rho)
        if ps > pk:  # shock on this side
            S = u + sgn * c * np.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pk + g2)
            behind = x > S if sgn < 0 else x < S
            out[:, j] = ((ps / pk + g1) / (g1 * ps / pk + 1.0) * rho, us, ps) if behind else (rho, u, pk)
        else:  # rarefaction on this side
            cs = c * (ps / pk) ** g2
            head, tail = u + sgn * c, us + sgn * cs
            if (sgn < 0 and x <= head) or (sgn > 0 and x >= head):
                out[:, j] = (rho, u, pk)
            elif (sgn < 0 and x >= tail) or (sgn > 0 and x <= tail):
                out[:, j] = (rho * (ps / pk) ** (1.0 / gamma), us, ps)
            else:  # inside the fan
                uf = 2.0 / (gamma + 1.0) * (-sgn * c + (gamma - 1.0) / 2.0 * u + x)
                cf = -sgn * (uf - x)
                out[:, j] = (rho * (cf / c) ** (2.0 / (gamma - 1.0)), uf, pk * (cf / c) ** (2.0 * gamma / (gamma - 1.0)))
    return out
