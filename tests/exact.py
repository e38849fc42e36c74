"""Closed-form solutions used to pin the oracle (no solver code here).

The dam-break problems are Riemann problems of the 1D shallow-water
equations with zero initial velocity (Sec. 6.3 of the paper refers to Toro's
book for the analytical solution).  The left rarefaction and the right shock
(wet bed, Stoker) or the single rarefaction reaching a dry front (Ritter)
follow from the Riemann invariants and the Rankine-Hugoniot relations.
"""
import math

import numpy as np


def stoker_star(hL, hR, g=9.81):
    """Middle state (h_m, u_m) and shock speed of the wet-bed dam break."""
    cL = math.sqrt(g * hL)

    def f(h):
        rare = 2.0 * (cL - math.sqrt(g * h))                             # u behind the rarefaction
        shock = (h - hR) * math.sqrt(g * (h + hR) / (2.0 * h * hR))       # u behind the shock
        return rare - shock

    lo, hi = hR, hL
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0:
            lo = mid
        else:
            hi = mid
    hm = 0.5 * (lo + hi)
    um = 2.0 * (cL - math.sqrt(g * hm))
    s = hm * um / (hm - hR)
    return hm, um, s


def stoker(x, t, x0, hL, hR, g=9.81):
    """Depth and velocity of the wet-bed dam break at time t."""
    hm, um, s = stoker_star(hL, hR, g)
    cL, cm = math.sqrt(g * hL), math.sqrt(g * hm)
    xi = (np.asarray(x, dtype=float) - x0) / t
    h = np.where(xi < -cL, hL, 0.0)
    u = np.zeros_like(xi)
    fan = (xi >= -cL) & (xi < um - cm)
    h = np.where(fan, (2 * cL - xi) ** 2 / (9 * g), h)
    u = np.where(fan, 2 * (xi + cL) / 3, u)
    mid = (xi >= um - cm) & (xi < s)
    h = np.where(mid, hm, h)
    u = np.where(mid, um, u)
    h = np.where(xi >= s, hR, h)
    return h, u


def ritter(x, t, x0, hL, g=9.81):
    """Dry-bed dam break: rarefaction from -sqrt(g hL) to the front at 2 sqrt(g hL)."""
    cL = math.sqrt(g * hL)
    xi = (np.asarray(x, dtype=float) - x0) / t
    h = np.where(xi < -cL, hL, (2 * cL - xi) ** 2 / (9 * g))
    h = np.where(xi >= 2 * cL, 0.0, h)
    return h


def manning_decay(u0, h, n, g, t):
    """Uniform flow slowed by Manning friction: du/dt = -g n^2 u|u| / h^(4/3)."""
    k = g * n * n / h ** (4.0 / 3.0)
    return u0 / (1.0 + k * abs(u0) * t)


def binned_profile(x, q, edges):
    """Mean of q over x-bins (y-average of a strip solution)."""
    idx = np.digitize(x, edges) - 1
    nb = len(edges) - 1
    ok = (idx >= 0) & (idx < nb)
    s = np.bincount(idx[ok], weights=np.asarray(q)[ok], minlength=nb)[:nb]
    c = np.bincount(idx[ok], minlength=nb)[:nb]
    return s / np.maximum(c, 1)
