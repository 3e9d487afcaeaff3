"""Exact solutions of 1D Riemann problems, used to pin the oracle's accuracy.

* Euler (ideal gas): pressure-function root of the star region and wave-fan
  sampling (Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics",
  Ch. 4), written out here from the gas-dynamics relations.
* Shallow water: left rarefaction / right shock dam break, middle depth from
  the Rankine-Hugoniot and Riemann-invariant relations.

No code is shared with the oracle or the CUDA library.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq


def euler_exact(rl, ul, pl, rr, ur, pr, gamma, xi):
    """Sample the exact Euler solution at similarity coordinates xi = (x-x0)/t.
    Returns (rho, u, p) arrays."""
    g = gamma
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)

    def f(p, rk, pk, ck):
        if p > pk:  # shock
            A = 2.0 / ((g + 1.0) * rk)
            B = (g - 1.0) / (g + 1.0) * pk
            return (p - pk) * math.sqrt(A / (p + B))
        return 2.0 * ck / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)

    def F(p):
        return f(p, rl, pl, cl) + f(p, rr, pr, cr) + (ur - ul)

    ps = brentq(F, 1e-12, 1e3 * max(pl, pr), xtol=1e-15, rtol=1e-15, maxiter=500)
    us = 0.5 * (ul + ur) + 0.5 * (f(ps, rr, pr, cr) - f(ps, rl, pl, cl))
    gm = (g - 1.0) / (g + 1.0)

    def star_rho(pk, rk):
        if ps > pk:
            return rk * ((ps / pk + gm) / (gm * ps / pk + 1.0))
        return rk * (ps / pk) ** (1.0 / g)

    rsl = star_rho(pl, rl)
    rsr = star_rho(pr, rr)
    out = np.zeros((3, len(xi)))
    for n, s in enumerate(xi):
        if s <= us:  # left of contact
            if ps > pl:  # left shock
                S = ul - cl * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                out[:, n] = (rl, ul, pl) if s <= S else (rsl, us, ps)
            else:  # left rarefaction
                head = ul - cl
                csl = cl * (ps / pl) ** ((g - 1) / (2 * g))
                tail = us - csl
                if s <= head:
                    out[:, n] = (rl, ul, pl)
                elif s >= tail:
                    out[:, n] = (rsl, us, ps)
                else:
                    u = 2.0 / (g + 1) * (cl + (g - 1) / 2 * ul + s)
                    c = 2.0 / (g + 1) * (cl + (g - 1) / 2 * (ul - s))
                    rho = rl * (c / cl) ** (2 / (g - 1))
                    out[:, n] = (rho, u, pl * (c / cl) ** (2 * g / (g - 1)))
        else:
            if ps > pr:  # right shock
                S = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                out[:, n] = (rr, ur, pr) if s >= S else (rsr, us, ps)
            else:  # right rarefaction
                head = ur + cr
                csr = cr * (ps / pr) ** ((g - 1) / (2 * g))
                tail = us + csr
                if s >= head:
                    out[:, n] = (rr, ur, pr)
                elif s <= tail:
                    out[:, n] = (rsr, us, ps)
                else:
                    u = 2.0 / (g + 1) * (-cr + (g - 1) / 2 * ur + s)
                    c = 2.0 / (g + 1) * (cr - (g - 1) / 2 * (ur - s))
                    rho = rr * (c / cr) ** (2 / (g - 1))
                    out[:, n] = (rho, u, pr * (c / cr) ** (2 * g / (g - 1)))
    return out


def sw_dambreak_exact(hl, hr, g, xi):
    """Dam break with zero velocities, hl > hr: 1-rarefaction, 2-shock.
    Returns (h, u) at similarity coordinates xi."""
    cl = math.sqrt(g * hl)

    def resid(hm):
        u_rar = 2.0 * (cl - math.sqrt(g * hm))
        u_sh = (hm - hr) * math.sqrt(0.5 * g * (hm + hr) / (hm * hr))
        return u_rar - u_sh

    hm = brentq(resid, hr, hl, xtol=1e-15, rtol=1e-15)
    um = 2.0 * (cl - math.sqrt(g * hm))
    cm = math.sqrt(g * hm)
    S = hm * um / (hm - hr)
    out = np.zeros((2, len(xi)))
    for n, s in enumerate(xi):
        if s <= -cl:
            out[:, n] = (hl, 0.0)
        elif s <= um - cm:
            c = (2.0 * cl - s) / 3.0
            out[:, n] = (c * c / g, s + c)
        elif s <= S:
            out[:, n] = (hm, um)
        else:
            out[:, n] = (hr, 0.0)
    return out
