"""Exact solution of the 1D Riemann problem for an ideal gas (oracle pin only).

Test infrastructure only. The Sod FOM (App. B) is pinned against this exact
self-similar solution: the star pressure solves
``f_L(p) + f_R(p) + (u_R - u_L) = 0`` with the shock (Rankine-Hugoniot) branch
of f_K for p > p_K and the rarefaction (isentropic) branch otherwise; the
solution at x/t is then sampled across the left wave, the contact and the right
wave. Written from the gas-dynamics relations (Toro, "Riemann Solvers and
Numerical Methods for Fluid Dynamics", ch. 4); the root is found with SciPy's
``brentq``.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq


def _f_branch(p, rho_k, p_k, c_k, gamma):
    if p > p_k:   # shock
        A = 2.0 / ((gamma + 1.0) * rho_k)
        B = (gamma - 1.0) / (gamma + 1.0) * p_k
        return (p - p_k) * math.sqrt(A / (p + B))
    # rarefaction
    return 2.0 * c_k / (gamma - 1.0) * ((p / p_k) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)


def star_state(left, right, gamma=1.4):
    """(p*, u*) of the Riemann problem with primitive states (rho, u, p)."""
    rL, uL, pL = left
    rR, uR, pR = right
    cL = math.sqrt(gamma * pL / rL)
    cR = math.sqrt(gamma * pR / rR)

    def fun(p):
        return _f_branch(p, rL, pL, cL, gamma) + _f_branch(p, rR, pR, cR, gamma) + (uR - uL)

    p_star = brentq(fun, 1e-14, 100.0 * max(pL, pR), xtol=1e-15, rtol=1e-15, maxiter=500)
    u_star = 0.5 * (uL + uR) + 0.5 * (_f_branch(p_star, rR, pR, cR, gamma)
                                      - _f_branch(p_star, rL, pL, cL, gamma))
    return p_star, u_star


def sample(left, right, xi, gamma=1.4):
    """Primitive (rho, u, p) arrays of the exact solution at similarity
    coordinates xi = (x - x0)/t."""
    rL, uL, pL = left
    rR, uR, pR = right
    cL = math.sqrt(gamma * pL / rL)
    cR = math.sqrt(gamma * pR / rR)
    ps, us = star_state(left, right, gamma)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    xi = np.asarray(xi, dtype=float)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    for k, s in enumerate(xi.flat):
        if s <= us:   # left of the contact
            if ps > pL:
                SL = uL - cL * math.sqrt((gamma + 1) / (2 * gamma) * ps / pL + (gamma - 1) / (2 * gamma))
                if s <= SL:
                    w = (rL, uL, pL)
                else:
                    w = (rL * (ps / pL + g1) / (g1 * ps / pL + 1.0), us, ps)
            else:
                cs = cL * (ps / pL) ** ((gamma - 1) / (2 * gamma))
                if s <= uL - cL:
                    w = (rL, uL, pL)
                elif s >= us - cs:
                    w = (rL * (ps / pL) ** (1.0 / gamma), us, ps)
                else:
                    uu = 2.0 / (gamma + 1) * (cL + 0.5 * (gamma - 1) * uL + s)
                    cc = 2.0 / (gamma + 1) * (cL + 0.5 * (gamma - 1) * (uL - s))
                    w = (rL * (cc / cL) ** (2.0 / (gamma - 1)), uu,
                         pL * (cc / cL) ** (2.0 * gamma / (gamma - 1)))
        else:         # right of the contact
            if ps > pR:
                SR = uR + cR * math.sqrt((gamma + 1) / (2 * gamma) * ps / pR + (gamma - 1) / (2 * gamma))
                if s >= SR:
                    w = (rR, uR, pR)
                else:
                    w = (rR * (ps / pR + g1) / (g1 * ps / pR + 1.0), us, ps)
            else:
                cs = cR * (ps / pR) ** ((gamma - 1) / (2 * gamma))
                if s >= uR + cR:
                    w = (rR, uR, pR)
                elif s <= us + cs:
                    w = (rR * (ps / pR) ** (1.0 / gamma), us, ps)
                else:
                    uu = 2.0 / (gamma + 1) * (-cR + 0.5 * (gamma - 1) * uR + s)
                    cc = 2.0 / (gamma + 1) * (cR - 0.5 * (gamma - 1) * (uR - s))
                    w = (rR * (cc / cR) ** (2.0 / (gamma - 1)), uu,
                         pR * (cc / cR) ** (2.0 * gamma / (gamma - 1)))
        rho.flat[k], u.flat[k], p.flat[k] = w
    return rho, u, p
