"""Textbook exact Riemann solver for the 1D Euler equations of a polytropic gas.

Test-only pin for the oracle, independent of it: the star pressure is found
by bisection on the monotone pressure function (not by the two-rarefaction
bound of Sec. 3.7), and the self-similar solution is sampled from the wave
structure (rarefaction fans, shocks, contact) in the usual way.
"""
from __future__ import annotations

import math

import numpy as np


def _fK(p, rho, pK, cK, gamma):
    if p > pK:
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pK
        return (p - pK) * math.sqrt(A / (p + B))
    return 2.0 * cK / (gamma - 1.0) * ((p / pK) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)


def star_pressure(left, right, gamma=1.4, rtol=1e-15):
    """Exact p* and u* for primitive states (rho, u, p); p* = 0 for vacuum."""
    rL, uL, pL = left
    rR, uR, pR = right
    cL = math.sqrt(gamma * pL / rL)
    cR = math.sqrt(gamma * pR / rR)

    def F(p):
        return _fK(p, rL, pL, cL, gamma) + _fK(p, rR, pR, cR, gamma) + uR - uL

    if F(0.0) >= 0.0:  # vacuum is generated
        return 0.0, None
    lo, hi = 0.0, max(pL, pR)
    while F(hi) < 0.0:
        hi *= 2.0
    for _ in range(400):
        mid = 0.5 * (lo + hi)
        if F(mid) < 0.0:
            lo = mid
        else:
            hi = mid
        if hi - lo <= rtol * hi:
            break
    p = 0.5 * (lo + hi)
    u = 0.5 * (uL + uR) + 0.5 * (_fK(p, rR, pR, cR, gamma) - _fK(p, rL, pL, cL, gamma))
    return p, u


def max_wave_speed(left, right, gamma=1.4):
    """max(|left wave speed|_neg, |right wave speed|_pos) of the exact solution."""
    rL, uL, pL = left
    rR, uR, pR = right
    cL = math.sqrt(gamma * pL / rL)
    cR = math.sqrt(gamma * pR / rR)
    p, _ = star_pressure(left, right, gamma)
    k = (gamma + 1.0) / (2.0 * gamma)
    sL = uL - cL * math.sqrt(1.0 + k * max(p - pL, 0.0) / pL)
    sR = uR + cR * math.sqrt(1.0 + k * max(p - pR, 0.0) / pR)
    return max(max(-sL, 0.0), max(sR, 0.0)), p


def sample(left, right, xi, gamma=1.4):
    """Primitive solution (rho, u, p) at similarity coordinates xi = x/t."""
    rL, uL, pL = left
    rR, uR, pR = right
    cL = math.sqrt(gamma * pL / rL)
    cR = math.sqrt(gamma * pR / rR)
    ps, us = star_pressure(left, right, gamma)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    out = np.empty((3, len(xi)))
    for q, s in enumerate(np.asarray(xi, dtype=float)):
        if s <= us:  # left of the contact
            if ps > pL:  # left shock
                SL = uL - cL * math.sqrt((gamma + 1) / (2 * gamma) * ps / pL + (gamma - 1) / (2 * gamma))
                if s <= SL:
                    r, u, p = rL, uL, pL
                else:
                    r = rL * (ps / pL + g1) / (g1 * ps / pL + 1.0)
                    u, p = us, ps
            else:  # left rarefaction
                cs = cL * (ps / pL) ** ((gamma - 1) / (2 * gamma))
                if s <= uL - cL:
                    r, u, p = rL, uL, pL
                elif s >= us - cs:
                    r, u, p = rL * (ps / pL) ** (1 / gamma), us, ps
                else:
                    u = 2 / (gamma + 1) * (cL + (gamma - 1) / 2 * uL + s)
                    c = 2 / (gamma + 1) * (cL + (gamma - 1) / 2 * (uL - s))
                    r = rL * (c / cL) ** (2 / (gamma - 1))
                    p = pL * (c / cL) ** (2 * gamma / (gamma - 1))
        else:
            if ps > pR:  # right shock
                SR = uR + cR * math.sqrt((gamma + 1) / (2 * gamma) * ps / pR + (gamma - 1) / (2 * gamma))
                if s >= SR:
                    r, u, p = rR, uR, pR
                else:
                    r = rR * (ps / pR + g1) / (g1 * ps / pR + 1.0)
                    u, p = us, ps
            else:
                cs = cR * (ps / pR) ** ((gamma - 1) / (2 * gamma))
                if s >= uR + cR:
                    r, u, p = rR, uR, pR
                elif s <= us + cs:
                    r, u, p = rR * (ps / pR) ** (1 / gamma), us, ps
                else:
                    u = 2 / (gamma + 1) * (-cR + (gamma - 1) / 2 * uR + s)
                    c = 2 / (gamma + 1) * (cR - (gamma - 1) / 2 * (uR - s))
                    r = rR * (c / cR) ** (2 / (gamma - 1))
                    p = pR * (c / cR) ** (2 * gamma / (gamma - 1))
        out[:, q] = (r, u, p)
    return out
