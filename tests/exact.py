"""Closed-form and textbook solutions used to pin the oracle (independent of it).

* exact Riemann solution of the Euler equations (Toro, "Riemann Solvers and Numerical Methods
  for Fluid Dynamics", ch. 4: pressure function, Newton iteration, wave sampling);
* linear MHD eigenmodes from the primitive-variable Jacobian (numerical eigen-decomposition);
* the spherically symmetric adiabatic wind with gravity (mass flux, entropy and Bernoulli
  constants, solved by bisection on the super-sonic branch).
"""
import math

import numpy as np


# --- exact Riemann solver (Euler, ideal gas) --------------------------------------------------
def _fk(p, rho, pk, a, g):
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        f = (p - pk) * math.sqrt(A / (p + B))
        df = math.sqrt(A / (B + p)) * (1.0 - (p - pk) / (2.0 * (B + p)))
    else:       # rarefaction
        f = 2.0 * a / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * a) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def riemann_star(wl, wr, g):
    rl, ul, pl = wl
    rr, ur, pr = wr
    al, ar = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    p = max(1e-8, 0.5 * (pl + pr))
    for _ in range(100):
        fl, dfl = _fk(p, rl, pl, al, g)
        fr, dfr = _fk(p, rr, pr, ar, g)
        pn = p - (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(pn, 1e-12)
        if abs(pn - p) < 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, al, g)
    fr, _ = _fk(p, rr, pr, ar, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def riemann_sample(wl, wr, g, s):
    """State (rho, u, p) at similarity coordinate s = x/t."""
    rl, ul, pl = wl
    rr, ur, pr = wr
    ps, us = riemann_star(wl, wr, g)
    al, ar = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    if s <= us:  # left of contact
        if ps > pl:
            sl = ul - al * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
            if s <= sl:
                return rl, ul, pl
            return rl * ((ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1)), us, ps
        shl = ul - al
        if s <= shl:
            return rl, ul, pl
        asl = al * (ps / pl) ** ((g - 1) / (2 * g))
        stl = us - asl
        if s > stl:
            return rl * (ps / pl) ** (1 / g), us, ps
        c = 2 / (g + 1) + (g - 1) / ((g + 1) * al) * (ul - s)
        return rl * c ** (2 / (g - 1)), 2 / (g + 1) * (al + (g - 1) / 2 * ul + s), pl * c ** (2 * g / (g - 1))
    if ps > pr:
        sr = ur + ar * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
        if s >= sr:
            return rr, ur, pr
        return rr * ((ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1)), us, ps
    shr = ur + ar
    if s >= shr:
        return rr, ur, pr
    asr = ar * (ps / pr) ** ((g - 1) / (2 * g))
    stR = us + asr
    if s <= stR:
        return rr * (ps / pr) ** (1 / g), us, ps
    c = 2 / (g + 1) - (g - 1) / ((g + 1) * ar) * (ur - s)
    return rr * c ** (2 / (g - 1)), 2 / (g + 1) * (-ar + (g - 1) / 2 * ur + s), pr * c ** (2 * g / (g - 1))


def riemann_profile(wl, wr, g, x, x0, t):
    out = np.array([riemann_sample(wl, wr, g, (xi - x0) / t) for xi in x])
    return out[:, 0], out[:, 1], out[:, 2]


# --- linear MHD waves -------------------------------------------------------------------------
def mhd_jacobian(w, g):
    """Primitive Jacobian along x for (rho, vx, vy, vz, p, By, Bz), Bx constant."""
    rho, vx, vy, vz, p, bx, by, bz = w
    A = np.zeros((7, 7))
    A[0, 0], A[0, 1] = vx, rho
    A[1, 1], A[1, 4], A[1, 5], A[1, 6] = vx, 1 / rho, by / rho, bz / rho
    A[2, 2], A[2, 5] = vx, -bx / rho
    A[3, 3], A[3, 6] = vx, -bx / rho
    A[4, 1], A[4, 4] = g * p, vx
    A[5, 1], A[5, 2], A[5, 5] = by, -bx, vx
    A[6, 1], A[6, 3], A[6, 6] = bz, -bx, vx
    return A


def mhd_modes(w, g):
    """Eigenvalues (sorted) and right eigenvectors [7][7] (columns) of the primitive Jacobian."""
    lam, R = np.linalg.eig(mhd_jacobian(w, g))
    lam, R = lam.real, R.real
    o = np.argsort(lam)
    return lam[o], R[:, o]


# --- spherical adiabatic wind -----------------------------------------------------------------
def wind_profile(r, r0, rho0, v0, p0, g, gm):
    """Super-sonic steady radial wind: rho v r^2, p / rho^g and
    v^2/2 + g/(g-1) p/rho - gm/r are constant. Returns (rho, v, p) at radii r."""
    mdot = rho0 * v0 * r0 * r0
    K = p0 / rho0 ** g
    E = 0.5 * v0 * v0 + g / (g - 1) * p0 / rho0 - gm / r0
    out = []
    for ri in np.atleast_1d(r):
        def F(v):
            rho = mdot / (v * ri * ri)
            return 0.5 * v * v + g / (g - 1) * K * rho ** (g - 1) - gm / ri - E
        # super-sonic root: bracket between the sonic point speed and a large speed
        lo, hi = 1e-6, 100.0
        # find the minimum of F (sonic point) on a log grid, then bisect above it
        vs = np.geomspace(lo, hi, 4000)
        fv = np.array([F(v) for v in vs])
        imin = int(np.argmin(fv))
        a, b = vs[imin], hi
        for _ in range(200):
            m = 0.5 * (a + b)
            if F(m) > 0:
                b = m
            else:
                a = m
        v = 0.5 * (a + b)
        rho = mdot / (v * ri * ri)
        out.append((rho, v, K * rho ** g))
    out = np.array(out)
    return out[:, 0], out[:, 1], out[:, 2]
