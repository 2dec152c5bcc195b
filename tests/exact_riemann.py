"""Exact Riemann solver for two stiffened gases (test tool, numpy float64).

Written from the textbook mathematics of the ideal-gas exact solver (Toro,
"Riemann Solvers and Numerical Methods for Fluid Dynamics", ch. 4) with
p -> p + p_inf on each side.  Independent of the oracle: it is used to pin
the oracle's fluid behaviour (shock tubes, the gas side of the solid impact).
"""
import math

import numpy as np


def _f(p, rho, pk, g, pinf):
    A = 2.0 / ((g + 1.0) * rho)
    B = (g - 1.0) / (g + 1.0) * (pk + pinf)
    c = math.sqrt(g * (pk + pinf) / rho)
    if p > pk:
        return (p - pk) * math.sqrt(A / (p + pinf + B))
    return 2.0 * c / (g - 1.0) * (((p + pinf) / (pk + pinf)) ** ((g - 1.0) / (2.0 * g)) - 1.0)


def star(L, R):
    """L, R: dicts rho, u, p, gamma, pinf.  Returns (p*, u*)."""
    def F(p):
        return _f(p, L["rho"], L["p"], L["gamma"], L["pinf"]) + \
            _f(p, R["rho"], R["p"], R["gamma"], R["pinf"]) + R["u"] - L["u"]
    lo = -min(L["pinf"], R["pinf"]) + 1e-12 * max(1.0, L["p"], R["p"])
    hi = max(L["p"], R["p"]) * 10 + 1.0
    while F(hi) < 0:
        hi *= 10
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if F(mid) > 0:
            hi = mid
        else:
            lo = mid
    ps = 0.5 * (lo + hi)
    us = 0.5 * (L["u"] + R["u"]) + 0.5 * (_f(ps, R["rho"], R["p"], R["gamma"], R["pinf"])
                                           - _f(ps, L["rho"], L["p"], L["gamma"], L["pinf"]))
    return ps, us


def sample(L, R, xi_arr):
    """Exact solution (rho, u, p, side) at similarity coordinates xi = (x - x0)/t."""
    ps, us = star(L, R)
    out = np.zeros((4, len(xi_arr)))
    for n, xi in enumerate(xi_arr):
        if xi <= us:
            K, sgn = L, -1.0
        else:
            K, sgn = R, 1.0
        g, pinf, rho, u, p = K["gamma"], K["pinf"], K["rho"], K["u"], K["p"]
        c = math.sqrt(g * (p + pinf) / rho)
        if ps > p:  # shock
            rs = rho * (((ps + pinf) / (p + pinf) + (g - 1) / (g + 1)) /
                        ((g - 1) / (g + 1) * (ps + pinf) / (p + pinf) + 1))
            S = u + sgn * c * math.sqrt((g + 1) / (2 * g) * (ps + pinf) / (p + pinf) + (g - 1) / (2 * g))
            if (sgn < 0 and xi <= S) or (sgn > 0 and xi >= S):
                out[:, n] = (rho, u, p, 0 if sgn < 0 else 1)
            else:
                out[:, n] = (rs, us, ps, 0 if sgn < 0 else 1)
        else:  # rarefaction
            rs = rho * ((ps + pinf) / (p + pinf)) ** (1 / g)
            cs = c * ((ps + pinf) / (p + pinf)) ** ((g - 1) / (2 * g))
            head = u + sgn * c
            tail = us + sgn * cs
            if (sgn < 0 and xi <= head) or (sgn > 0 and xi >= head):
                out[:, n] = (rho, u, p, 0 if sgn < 0 else 1)
            elif (sgn < 0 and xi >= tail) or (sgn > 0 and xi <= tail):
                out[:, n] = (rs, us, ps, 0 if sgn < 0 else 1)
            else:
                cc = 2 / (g + 1) * (c - sgn * (g - 1) / 2 * (u - xi))
                uu = 2 / (g + 1) * (-sgn * c + (g - 1) / 2 * u + xi)
                rr = rho * (cc / c) ** (2 / (g - 1))
                pp = (p + pinf) * (cc / c) ** (2 * g / (g - 1)) - pinf
                out[:, n] = (rr, uu, pp, 0 if sgn < 0 else 1)
    return out
