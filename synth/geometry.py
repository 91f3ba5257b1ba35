"""Cell-kind masks of the paper's geometries (uint8, shape (ny, nx))."""
from __future__ import annotations

import math

import numpy as np

FLUID, SOLID, WALL = 0, 1, 2


def cylinder_mask(nx, ny, xc, yc, diameter):
    """Cylinder of Fig. 2: node (x, y) is solid iff (x-xc)^2 + (y-yc)^2 <= (D/2)^2."""
    y, x = np.mgrid[0:ny, 0:nx]
    r2 = (x - xc) ** 2 + (y - yc) ** 2
    kind = np.zeros((ny, nx), dtype=np.uint8)
    kind[r2 <= (diameter / 2.0) ** 2] = SOLID
    return kind


def add_walls(kind):
    """Channel walls: rows 0 and ny-1 become uncounted solid rows (they take
    precedence over anything else on those rows)."""
    out = kind.copy()
    out[0, :] = WALL
    out[-1, :] = WALL
    return out


# Appendix A: closed-trailing-edge NACA four-digit thickness law for t = 0.12
_NACA_SCALE = 0.594689181
_NACA_COEF = (0.298222773, -0.127125232, -0.357907906, 0.291984971, -0.105174606)


def naca0012_half_thickness(xc):
    """Half thickness y_t(x) for chordwise x in [0, 1] (Appendix A)."""
    xc = np.asarray(xc, dtype=np.float64)
    a0, a1, a2, a3, a4 = _NACA_COEF
    return _NACA_SCALE * (a0 * np.sqrt(xc) + a1 * xc + a2 * xc ** 2 + a3 * xc ** 3 + a4 * xc ** 4)


def naca0012_mask(nx, ny, chord, x_le, y_mid, aoa_deg):
    """Staircase NACA0012 mask: leading edge at (x_le, y_mid), rotated nose-up
    by ``aoa_deg`` about the quarter chord; node solid iff, in the airfoil's
    frame, 0 <= x' <= 1 and |y'| <= y_t(x')."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    xq = x_le + 0.25 * chord
    a = math.radians(aoa_deg)
    dx, dy = x - xq, y - y_mid
    # rotate the lattice into the chord frame (nose-up angle of attack)
    xr = dx * math.cos(a) - dy * math.sin(a)
    yr = dx * math.sin(a) + dy * math.cos(a)
    xp = xr / chord + 0.25
    yp = yr / chord
    inside = (xp >= 0.0) & (xp <= 1.0)
    yt = naca0012_half_thickness(np.clip(xp, 0.0, 1.0))
    kind = np.zeros((ny, nx), dtype=np.uint8)
    kind[inside & (np.abs(yp) <= yt)] = SOLID
    return kind
