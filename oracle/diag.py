"""Measurements of Secs. 3-4 of arXiv:2009.12584 on oracle fields, in plain
numpy and Python loops, for comparison with the library's on-device
diagnostics.

TEST INFRASTRUCTURE, like the rest of ``oracle``: only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
it; it imports nothing from the CUDA library's package.

Definitions (the readings of the paper's text that the library states in its
header):
  - contour points: where rho^A - level changes sign along a grid edge
    joining two fluid nodes (x, y)-(x+1, y) or (x, y)-(x, y+1), no periodic
    wrap; the point is placed by linear interpolation of rho^A;
  - circle: the algebraic least-squares (Kasa) fit, the circle
    x^2 + y^2 = A x + B y + C closest in the least-squares sense;
  - contact angle: cos(theta) = -h / R, h the signed distance from the wall
    line to the circle centre, positive on the fluid side (left-hand normal
    (-sin b, cos b) of the wall direction (cos b, sin b)); points within
    ``exclude`` of the wall line are not fitted (Sec. 3.2);
  - sliding velocity: centre-of-mass velocity with weight
    w = max(rho^A - rho_out, 0) over fluid nodes, projected on a tangent
    (Sec. 3.1);
  - bridge radius: on one column, the distance from the halfway wall below
    the first fluid node to where rho^A first drops through ``level``
    (Sec. 4);
  - max |u| over fluid nodes (Sec. 4, spurious currents).
"""
from __future__ import annotations

import math

import numpy as np


def _sgn(v: float) -> int:
    return int(v > 0) - int(v < 0)


def contour_points(rhoA, mask, level=0.5):
    """List of (x, y) crossings of ``level`` on edges between fluid nodes."""
    rhoA = np.asarray(rhoA, float)
    fluid = np.asarray(mask) == 0
    ny, nx = rhoA.shape
    pts = []
    for y in range(ny):
        for x in range(nx):
            if not fluid[y, x]:
                continue
            a = rhoA[y, x] - level
            if x + 1 < nx and fluid[y, x + 1]:
                b = rhoA[y, x + 1] - level
                if _sgn(a) != _sgn(b) and a != b:
                    pts.append((x + a / (a - b), float(y)))
            if y + 1 < ny and fluid[y + 1, x]:
                b = rhoA[y + 1, x] - level
                if _sgn(a) != _sgn(b) and a != b:
                    pts.append((float(x), y + a / (a - b)))
    return pts


def kasa_fit(pts):
    """(xc, yc, R) of the algebraic least-squares circle through ``pts``:
    minimise sum (x^2 + y^2 - A x - B y - C)^2, then xc = A/2, yc = B/2,
    R^2 = C + xc^2 + yc^2. The least-squares problem is solved by
    numpy's lstsq (SVD)."""
    p = np.asarray(pts, float)
    x, y = p[:, 0], p[:, 1]
    M = np.stack([x, y, np.ones_like(x)], axis=1)
    (A, B, C), *_ = np.linalg.lstsq(M, x * x + y * y, rcond=None)
    xc, yc = A / 2.0, B / 2.0
    return xc, yc, math.sqrt(C + xc * xc + yc * yc)


def wall_normal(wall_angle_deg):
    b = math.radians(wall_angle_deg)
    return -math.sin(b), math.cos(b)


def contact_angle(rhoA, mask, wall_point, wall_angle_deg, exclude=3.0, level=0.5, box=None):
    """(theta in degrees, (xc, yc, R), number of fitted points)."""
    nxw, nyw = wall_normal(wall_angle_deg)
    keep = []
    for (px, py) in contour_points(rhoA, mask, level):
        dist = (px - wall_point[0]) * nxw + (py - wall_point[1]) * nyw
        if not dist > exclude:
            continue
        if box is not None and not (box[0] <= px <= box[1] and box[2] <= py <= box[3]):
            continue
        keep.append((px, py))
    xc, yc, R = kasa_fit(keep)
    h = (xc - wall_point[0]) * nxw + (yc - wall_point[1]) * nyw
    c = max(-1.0, min(1.0, -h / R))
    return math.degrees(math.acos(c)), (xc, yc, R), len(keep)


def weighted_com(rhoA, u, mask, rho_out):
    """(sum w, centre of mass (x, y), mean velocity (u_x, u_y)) with
    w = max(rho^A - rho_out, 0) over fluid nodes."""
    rhoA = np.asarray(rhoA, float)
    fluid = np.asarray(mask) == 0
    ny, nx = rhoA.shape
    W = Wx = Wy = Wu = Wv = 0.0
    for y in range(ny):
        for x in range(nx):
            if not fluid[y, x]:
                continue
            w = max(rhoA[y, x] - rho_out, 0.0)
            W += w
            Wx += w * x
            Wy += w * y
            Wu += w * u[0][y, x]
            Wv += w * u[1][y, x]
    return W, (Wx / W, Wy / W), (Wu / W, Wv / W)


def sliding_velocity(rhoA, u, mask, rho_out, tangent):
    _, _, (vx, vy) = weighted_com(rhoA, u, mask, rho_out)
    return vx * tangent[0] + vy * tangent[1]


def max_speed(u, mask):
    fluid = np.asarray(mask) == 0
    s = np.sqrt(np.asarray(u[0]) ** 2 + np.asarray(u[1]) ** 2)
    return float(s[fluid].max())


def bridge_radius(rhoA, x_col, y0, level=0.5):
    """Distance from the halfway wall (y0 - 1/2) to the first point above
    y0 on column ``x_col`` where rho^A drops through ``level``; 0 while
    rho^A(x_col, y0) < level; the top of the grid if it never drops."""
    col = np.asarray(rhoA, float)[:, x_col]
    if col[y0] < level:
        return 0.0
    y = y0
    while y + 1 < len(col):
        if col[y + 1] < level:
            t = (col[y] - level) / (col[y] - col[y + 1])
            return (y + t) - (y0 - 0.5)
        y += 1
    return len(col) - (y0 - 0.5)
