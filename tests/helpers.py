"""Shared test helpers: grids for the pins and plain numpy utilities (no solver arithmetic)."""
import math

import numpy as np

from paper_2501_15923_gb300 import inputs as I


def cart_grid(n1, n2=1, n3=1, L=(1.0, 1.0, 1.0), bc=(I.BC_PERIODIC,) * 6):
    return I.Grid(n1, n2, n3, geometry=I.GEOM_CARTESIAN, stretch=0, x1min=0.0, x1max=L[0],
                  x2min=0.0, x2max=L[1], x3min=0.0, x3max=L[2], bc=tuple(bc))


def sph_grid(n1, n2, n3, bc, r=(0.1, 2.0), th=(math.radians(30), math.radians(150)),
             ph=(0.0, 2 * math.pi), stretch=1):
    return I.Grid(n1, n2, n3, geometry=I.GEOM_SPHERICAL, stretch=stretch, x1min=r[0], x1max=r[1],
                  x2min=th[0], x2max=th[1], x3min=ph[0], x3max=ph[1], bc=tuple(bc))


def opts(**kw):
    o = I.Options()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def edges(g, d):
    n = (g.n1, g.n2, g.n3)[d]
    lo, hi = [(g.x1min, g.x1max), (g.x2min, g.x2max), (g.x3min, g.x3max)][d]
    i = np.arange(-2, n + 3)
    if d == 0 and g.geometry == I.GEOM_SPHERICAL and g.stretch:
        return lo * (hi / lo) ** (i / n)
    return lo + i * ((hi - lo) / n)


def centres(g, d):
    e = edges(g, d)
    return 0.5 * (e[:-1] + e[1:])


def l1(a):
    return float(np.mean(np.abs(a)))
