"""Exact Riemann solver for two stiffened-gas materials separated by a contact.

Textbook solution (Toro, "Riemann Solvers and Numerical Methods for Fluid
Dynamics", ch. 4) written for the stiffened-gas EOS p + pinf = (gamma-1) rho e
- gamma pinf + pinf, i.e. with p replaced by p + pinf in every wave relation;
each side keeps its own (gamma, pinf).  Used as the reference curve for the
two-fluid shock tube without heat conduction (paper Sec. 4.2, test without
heat conduction).  Independent of the oracle: nothing here is shared with it.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq


class Side:
    def __init__(self, rho, u, p, gamma, pinf):
        self.rho, self.u, self.p, self.g, self.pi = rho, u, p, gamma, pinf
        self.c = math.sqrt(gamma * (p + pinf) / rho)

    def f(self, p):
        g, pi, pk = self.g, self.pi, self.p
        if p > pk:
            A = 2.0 / ((g + 1.0) * self.rho)
            B = (g - 1.0) / (g + 1.0) * (pk + pi)
            return (p - pk) * math.sqrt(A / (p + pi + B))
        return 2.0 * self.c / (g - 1.0) * (((p + pi) / (pk + pi)) ** ((g - 1.0) / (2.0 * g)) - 1.0)


def solve(L: Side, R: Side):
    """Star pressure and velocity."""
    def fun(p):
        return L.f(p) + R.f(p) + R.u - L.u

    lo = -min(L.pi, R.pi) + 1e-9 * max(1.0, L.p, R.p)
    hi = 10.0 * max(L.p + L.pi, R.p + R.pi)
    ps = brentq(fun, lo, hi, xtol=1e-14 * hi, rtol=1e-15, maxiter=500)
    us = 0.5 * (L.u + R.u) + 0.5 * (R.f(ps) - L.f(ps))
    return ps, us


def _sample_side(K: Side, ps, us, S, sign):
    """State at x/t = S on side K (sign = -1 left, +1 right of the contact)."""
    g, pi = K.g, K.pi
    pr = (ps + pi) / (K.p + pi)
    if ps > K.p:  # shock
        Ssh = K.u + sign * K.c * math.sqrt((g + 1.0) / (2.0 * g) * pr + (g - 1.0) / (2.0 * g))
        if sign * (S - Ssh) >= 0.0:
            return K.rho, K.u, K.p
        rs = K.rho * (pr + (g - 1.0) / (g + 1.0)) / ((g - 1.0) / (g + 1.0) * pr + 1.0)
        return rs, us, ps
    cs = K.c * pr ** ((g - 1.0) / (2.0 * g))
    Shead = K.u + sign * K.c
    Stail = us + sign * cs
    if sign * (S - Shead) >= 0.0:
        return K.rho, K.u, K.p
    if sign * (S - Stail) <= 0.0:
        return K.rho * pr ** (1.0 / g), us, ps
    # inside the fan
    u = 2.0 / (g + 1.0) * (-sign * K.c + (g - 1.0) / 2.0 * K.u + S)
    c = 2.0 / (g + 1.0) * (K.c - sign * (g - 1.0) / 2.0 * (K.u - S))
    rho = K.rho * (c / K.c) ** (2.0 / (g - 1.0))
    p = (K.p + pi) * (c / K.c) ** (2.0 * g / (g - 1.0)) - pi
    return rho, u, p


def sample(L: Side, R: Side, x: np.ndarray, x0: float, t: float):
    """(rho, u, p, side) at positions x, time t, initial jump at x0."""
    ps, us = solve(L, R)
    out = np.zeros((4, x.size))
    for i, xi in enumerate(x):
        S = (xi - x0) / t
        if S <= us:
            r, u, p = _sample_side(L, ps, us, S, -1.0)
            side = 0
        else:
            r, u, p = _sample_side(R, ps, us, S, +1.0)
            side = 1
        out[:, i] = (r, u, p, side)
    return out, ps, us
