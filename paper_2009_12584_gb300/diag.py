"""Host-side measurements on density/velocity fields (numpy).

These read fields that the library (or the oracle) has already produced:
the contact angle of a sessile droplet by a circle fit to the rho^A = 0.5
contour (Sec. 3.2), the droplet's centre-of-mass sliding velocity along a
wall (Sec. 3.1) and the bridge radius of two coalescing droplets (Sec. 4).
They are measurements, not part of the time step.
"""
from __future__ import annotations

import math

import numpy as np


def contour_points(rhoA: np.ndarray, mask: np.ndarray, level: float = 0.5) -> np.ndarray:
    """Points where rho^A crosses ``level`` on grid edges joining two fluid
    nodes, by linear interpolation. Returns an (n, 2) array of (x, y)."""
    pts = []
    fluid = mask == 0
    d = rhoA - level
    # horizontal edges (x, y) - (x + 1, y)
    a, b = d[:, :-1], d[:, 1:]
    ok = fluid[:, :-1] & fluid[:, 1:] & (np.sign(a) != np.sign(b)) & (a != b)
    yy, xx = np.nonzero(ok)
    t = a[ok] / (a[ok] - b[ok])
    pts.append(np.stack([xx + t, yy.astype(float)], axis=1))
    # vertical edges (x, y) - (x, y + 1)
    a, b = d[:-1, :], d[1:, :]
    ok = fluid[:-1, :] & fluid[1:, :] & (np.sign(a) != np.sign(b)) & (a != b)
    yy, xx = np.nonzero(ok)
    t = a[ok] / (a[ok] - b[ok])
    pts.append(np.stack([xx.astype(float), yy + t], axis=1))
    return np.concatenate(pts, axis=0)


def fit_circle(pts: np.ndarray):
    """Algebraic least-squares (Kasa) circle fit: (xc, yc, R)."""
    x, y = pts[:, 0], pts[:, 1]
    A = np.stack([x, y, np.ones_like(x)], axis=1)
    rhs = x * x + y * y
    (a, b, c), *_ = np.linalg.lstsq(A, rhs, rcond=None)
    xc, yc = a / 2, b / 2
    return xc, yc, math.sqrt(c + xc * xc + yc * yc)


def contact_angle(rhoA: np.ndarray, mask: np.ndarray, wall_point, wall_angle_deg: float,
                  exclude: float = 3.0, level: float = 0.5, select=None) -> float:
    """Contact angle (degrees, measured through the A phase) of a droplet
    sitting on the straight wall through ``wall_point`` inclined at
    ``wall_angle_deg``; the fluid lies on the wall's left-hand normal side.
    Contour points closer than ``exclude`` to the wall are dropped; a circle
    is fitted to the rest and cos(theta) = -h / R with h the signed distance
    from the wall to the circle centre (positive on the fluid side)."""
    pts = contour_points(rhoA, mask, level)
    b = math.radians(wall_angle_deg)
    nrm = np.array([-math.sin(b), math.cos(b)])
    p0 = np.asarray(wall_point, float)
    dist = (pts - p0) @ nrm
    keep = dist > exclude
    if select is not None:
        keep &= select(pts)
    xc, yc, R = fit_circle(pts[keep])
    h = (np.array([xc, yc]) - p0) @ nrm
    c = max(-1.0, min(1.0, -h / R))
    return math.degrees(math.acos(c))


def com_velocity(rhoA: np.ndarray, u: np.ndarray, rho_out: float, tangent) -> float:
    """Centre-of-mass velocity of the A droplet along ``tangent``, weighted
    by max(rho^A - rho_out, 0) (a continuous weight, so that no threshold
    flips between runs in different precisions)."""
    w = np.maximum(rhoA - rho_out, 0.0)
    t = np.asarray(tangent, float)
    return float(((w * u[0]).sum() * t[0] + (w * u[1]).sum() * t[1]) / w.sum())


def com_position(rhoA: np.ndarray, rho_out: float):
    w = np.maximum(rhoA - rho_out, 0.0)
    ny, nx = rhoA.shape
    X = (w * np.arange(nx)[None, :]).sum() / w.sum()
    Y = (w * np.arange(ny)[:, None]).sum() / w.sum()
    return float(X), float(Y)


def bridge_radius(rhoA: np.ndarray, x_col: int, y_first_fluid: int,
                  level: float = 0.5) -> float:
    """Bridge radius b of Sec. 4 on the symmetry column ``x_col``: the
    distance from the halfway wall (half a node below ``y_first_fluid``, the
    first fluid node above the surface) to the first point above it where
    rho^A drops through ``level`` (linear interpolation); 0 while the fluid
    next to the wall is below ``level``."""
    col = rhoA[:, x_col]
    y = y_first_fluid
    if col[y] < level:
        return 0.0
    while y + 1 < len(col) and col[y + 1] >= level:
        y += 1
    if y + 1 >= len(col):
        return float(len(col) - (y_first_fluid - 0.5))
    t = (col[y] - level) / (col[y] - col[y + 1])
    return float(y + t - (y_first_fluid - 0.5))
