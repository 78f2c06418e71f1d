"""Pins of the oracle's measurement functions (oracle/diag.py) against
closed forms: exact circles, linear fields, uniform velocity fields and
constructed column profiles. Each pin is chosen so that a plausible
mistake (a wrong normal sign, a dropped interpolation term, an off-by-one
halfway wall, a transposed axis) fails it."""
import math

import numpy as np
import pytest

from oracle import diag


def test_kasa_fit_exact_circle():
    rng = np.random.default_rng(3)
    xc, yc, R = 3.1, -2.4, 17.3
    t = rng.uniform(0.2, 2.9, 40)  # an arc, not the whole circle
    pts = np.stack([xc + R * np.cos(t), yc + R * np.sin(t)], axis=1)
    fx, fy, fR = diag.kasa_fit(pts)
    assert abs(fx - xc) < 1e-9 and abs(fy - yc) < 1e-9 and abs(fR - R) < 1e-9


def test_kasa_fit_translation_invariant():
    rng = np.random.default_rng(4)
    pts = rng.normal(size=(30, 2)) * 5.0 + np.array([10.0, 20.0])
    a = diag.kasa_fit(pts)
    b = diag.kasa_fit(pts + np.array([700.0, -350.0]))
    assert abs(b[0] - 700.0 - a[0]) < 1e-8 and abs(b[1] + 350.0 - a[1]) < 1e-8 and abs(b[2] - a[2]) < 1e-8


def test_contour_points_linear_field():
    ny, nx = 6, 20
    x = np.arange(nx)[None, :].repeat(ny, 0).astype(float)
    rho = 0.5 + 0.1 * (x - 7.3)  # crosses 0.5 at x = 7.3 on every row, never along y
    mask = np.zeros((ny, nx), np.uint8)
    pts = diag.contour_points(rho, mask)
    assert len(pts) == ny
    for (px, py), y in zip(sorted(pts, key=lambda p: p[1]), range(ny)):
        assert abs(px - 7.3) < 1e-12 and py == y
    # an edge touching a solid node carries no crossing
    mask[2, 8] = 1
    assert len(diag.contour_points(rho, mask)) == ny - 1
    # the same field along y crosses on vertical edges
    pts = diag.contour_points(rho.T.copy(), np.zeros((nx, ny), np.uint8))
    assert len(pts) == ny and all(abs(py - 7.3) < 1e-12 for _, py in pts)


def _droplet(nx, ny, xc, yc, R, width=2.0):
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    r = np.hypot(x - xc, y - yc)
    return 0.5 - 0.5 * np.tanh((r - R) / width)


@pytest.mark.parametrize("h", [-15.0, 0.0, 10.0])
def test_contact_angle_of_a_cut_circle(h):
    # wall: row 0 solid, halfway plane y = 0.5; circle of radius R whose
    # centre is h above that plane: theta = acos(-h / R)
    nx, ny, R = 140, 80, 40.0
    mask = np.zeros((ny, nx), np.uint8)
    mask[0, :] = 1
    rho = _droplet(nx, ny, 70.0, 0.5 + h, R)
    th, (xc, yc, fR), n = diag.contact_angle(rho, mask, (0.0, 0.5), 0.0)
    assert n > 50
    assert abs(th - math.degrees(math.acos(-h / R))) < 0.3
    assert abs(fR - R) < 0.1 and abs(xc - 70.0) < 0.05 and abs(yc - (0.5 + h)) < 0.1


def test_contact_angle_inclined_wall_and_box():
    # wall through (0, 0.5) at 30 degrees: fluid on the side of (-sin, cos)
    nx, ny, R, b = 160, 120, 30.0, math.radians(30.0)
    nrm = np.array([-math.sin(b), math.cos(b)])
    foot = np.array([80.0, 0.5 + 80.0 * math.tan(b)])
    h = 12.0
    c = foot + h * nrm
    mask = np.zeros((ny, nx), np.uint8)
    rho = _droplet(nx, ny, c[0], c[1], R)
    th, _, _ = diag.contact_angle(rho, mask, (0.0, 0.5), 30.0)
    assert abs(th - math.degrees(math.acos(-h / R))) < 0.3
    # a second droplet far away is removed by the box
    rho2 = np.maximum(rho, _droplet(nx, ny, 140.0, 105.0, 8.0))
    box = (c[0] - 45, c[0] + 45, c[1] - 45, c[1] + 45)
    th2, _, _ = diag.contact_angle(rho2, mask, (0.0, 0.5), 30.0, box=box)
    assert abs(th2 - th) < 1e-12
    th3, _, _ = diag.contact_angle(rho2, mask, (0.0, 0.5), 30.0)
    assert abs(th3 - th) > 1.0  # without the box the second droplet spoils the fit


def test_weighted_com_and_sliding_velocity():
    ny, nx = 10, 12
    rng = np.random.default_rng(5)
    rho = rng.uniform(0.0, 1.0, (ny, nx))
    mask = np.zeros((ny, nx), np.uint8)
    mask[0, :] = 1
    u = (np.full((ny, nx), 0.01), np.full((ny, nx), -0.02))
    W, (X, Y), (vx, vy) = diag.weighted_com(rho, u, mask, 0.3)
    w = np.maximum(rho - 0.3, 0) * (mask == 0)
    yy, xx = np.mgrid[0:ny, 0:nx]
    assert abs(W - w.sum()) < 1e-12
    assert abs(X - (w * xx).sum() / w.sum()) < 1e-12 and abs(Y - (w * yy).sum() / w.sum()) < 1e-12
    assert abs(vx - 0.01) < 1e-15 and abs(vy + 0.02) < 1e-15
    t = (math.cos(0.3), math.sin(0.3))
    assert abs(diag.sliding_velocity(rho, u, mask, 0.3, t) - (0.01 * t[0] - 0.02 * t[1])) < 1e-15


def test_max_speed_ignores_solid():
    u = (np.array([[3.0, 0.1], [0.0, 0.0]]), np.array([[4.0, 0.0], [0.2, 0.0]]))
    mask = np.array([[1, 0], [0, 0]], np.uint8)
    assert diag.max_speed(u, mask) == pytest.approx(0.2, abs=1e-15)
    mask[0, 0] = 0
    assert diag.max_speed(u, mask) == 5.0


def test_bridge_radius_column():
    ny, nx = 30, 5
    rho = np.zeros((ny, nx))
    y0 = 3
    rho[y0:, 2] = np.clip(1.0 - 0.1 * (np.arange(y0, ny) - y0), 0, None)  # 0.5 at y0 + 5
    assert diag.bridge_radius(rho, 2, y0) == pytest.approx(5.5, abs=1e-12)
    assert diag.bridge_radius(rho, 1, y0) == 0.0  # below the level next to the wall
    rho[:, 4] = 1.0
    assert diag.bridge_radius(rho, 4, y0) == pytest.approx(ny - (y0 - 0.5))
