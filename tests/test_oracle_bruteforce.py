"""Brute-force pins of the oracle on tiny grids.

Every quantity is written out here a second time with named neighbours (east,
north-east, ...), the constants of Eqs. 2-4 expanded for c_s^2 = 1/3, and the
D2Q25 classes listed by hand, then compared with the oracle's loops to
1e-14. Grids are padded with two solid layers so that np.roll never wraps
real data into a non-periodic stencil."""
import numpy as np
import pytest

import oracle
from paper_2009_12584_gb300 import inputs

G = 3.0


def at(a, dx, dy):
    """Value of field a at (x + dx, y + dy), periodic wrap."""
    return np.roll(a, (-dy, -dx), axis=(-2, -1))


# D2Q9 in the oracle's order: 0 rest, 1 E, 2 N, 3 W, 4 S, 5 NE, 6 NW, 7 SW, 8 SE
E, N, W_, S_ = (1, 0), (0, 1), (-1, 0), (0, -1)
NE, NW, SW, SE = (1, 1), (-1, 1), (-1, -1), (1, -1)


def sc_sum(val, fluid):
    """sum_i w_i c_i fluid(x+c_i) val(x+c_i), written out per neighbour."""
    def g(d):
        return at(fluid, *d) * at(val, *d)
    sx = (g(E) - g(W_)) / 9 + (g(NE) - g(NW) - g(SW) + g(SE)) / 36
    sy = (g(N) - g(S_)) / 9 + (g(NE) + g(NW) - g(SW) - g(SE)) / 36
    return sx, sy


def d2q25_average(rho, fluid):
    """Eq. 8 average with the D2Q25 classes written out."""
    ring1 = [(1, 0), (0, 1), (-1, 0), (0, -1)]
    diag1 = [(1, 1), (-1, 1), (-1, -1), (1, -1)]
    axis2 = [(2, 0), (0, 2), (-2, 0), (0, -2)]
    knight = [(2, 1), (1, 2), (-1, 2), (-2, 1), (-2, -1), (-1, -2), (1, -2), (2, -1)]
    corner2 = [(2, 2), (-2, 2), (-2, -2), (2, -2)]
    num = np.zeros_like(rho)
    den = np.zeros_like(rho)
    for cls, wt in ((ring1, 4 / 21), (diag1, 4 / 45), (axis2, 1 / 60), (knight, 2 / 315),
                    (corner2, 1 / 5040)):
        for d in cls:
            num += wt * at(fluid, *d) * at(rho, *d)
            den += wt * at(fluid, *d)
    return num / np.where(den > 0, den, 1.0)


def reference_step(f, mask, bc, tau, Gs, chi, rho_s, pairing):
    """One step of Eqs. 1-8 written out independently of the oracle."""
    fluid = 1.0 - mask
    solid = mask.astype(float)
    rho = f.sum(axis=1) * fluid
    iface = solid * ((at(fluid, *E) + at(fluid, *N) + at(fluid, *W_) + at(fluid, *S_)
                      + at(fluid, *NE) + at(fluid, *NW) + at(fluid, *SW) + at(fluid, *SE)) > 0)
    rt = np.zeros_like(rho)
    if bc == oracle.BC_VIRTUAL_AVG:
        for s in range(2):
            rt[s] = chi[s] * d2q25_average(rho[s], fluid) * iface
    F = np.zeros((2, 2) + mask.shape)
    for s in range(2):
        o = 1 - s
        c = s if pairing == oracle.PAIR_SELF else o
        ax, ay = sc_sum(rho[o], fluid)
        if bc == oracle.BC_MARTYS_CHEN:
            bx, by = sc_sum(np.ones_like(rho[0]), solid)
        elif bc == oracle.BC_LLKC:
            vx, vy = sc_sum(np.ones_like(rho[0]), solid)
            bx, by = vx * rho[c], vy * rho[c]
        elif bc == oracle.BC_VIRTUAL_AVG:
            bx, by = sc_sum(rt[c], solid)
        else:
            vx, vy = sc_sum(np.ones_like(rho[0]), solid)
            bx, by = vx * rho_s[c], vy * rho_s[c]
        F[s, 0] = (-rho[s] * (G * ax + Gs[s] * bx)) * fluid
        F[s, 1] = (-rho[s] * (G * ay + Gs[s] * by)) * fluid
    # Eq. 3 with the D2Q9 velocities written out
    jx = sum(f[s, 1] - f[s, 3] + f[s, 5] - f[s, 6] - f[s, 7] + f[s, 8] for s in range(2))
    jy = sum(f[s, 2] - f[s, 4] + f[s, 5] + f[s, 6] - f[s, 7] - f[s, 8] for s in range(2))
    rsum = np.where(fluid > 0, rho[0] + rho[1], 1.0)
    ux = (jx + 0.5 * (F[0, 0] + F[1, 0])) / rsum * fluid
    uy = (jy + 0.5 * (F[0, 1] + F[1, 1])) / rsum * fluid
    cx = [0, 1, 0, -1, 0, 1, -1, -1, 1]
    cy = [0, 0, 1, 0, -1, 1, 1, -1, -1]
    w = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
    fpost = np.zeros_like(f)
    usq = ux * ux + uy * uy
    for s in range(2):
        for i in range(9):
            cu = cx[i] * ux + cy[i] * uy
            feq = rho[s] * w[i] * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * usq)
            src = w[i] * (1 - 0.5 / tau[s]) * (
                (3 * cx[i] + 9 * cu * cx[i] - 3 * ux) * F[s, 0]
                + (3 * cy[i] + 9 * cu * cy[i] - 3 * uy) * F[s, 1])
            fpost[s, i] = (f[s, i] - (f[s, i] - feq) / tau[s] + src) * fluid
    opp = [0, 3, 4, 1, 2, 7, 8, 5, 6]
    fnew = np.zeros_like(f)
    for s in range(2):
        for i in range(9):
            upstream_fluid = at(fluid, -cx[i], -cy[i])
            pulled = at(fpost[s, i], -cx[i], -cy[i])
            fnew[s, i] = (upstream_fluid * pulled + (1 - upstream_fluid) * fpost[s, opp[i]]) * fluid
    return rho, rt, F, np.stack([ux, uy]), fnew


CASES = [
    # (name, bc, Gs, chi, rho_s, pairing)
    ("mc", oracle.BC_MARTYS_CHEN, (-0.3, 0.3), (1, 1), (0, 0), oracle.PAIR_CROSS),
    ("mc_asym", oracle.BC_MARTYS_CHEN, (0.2, 0.5), (1, 1), (0, 0), oracle.PAIR_CROSS),
    ("llkc", oracle.BC_LLKC, (-0.5, 0.5), (1, 1), (0, 0), oracle.PAIR_CROSS),
    ("llkc_self", oracle.BC_LLKC, (-0.5, 0.4), (1, 1), (0, 0), oracle.PAIR_SELF),
    ("improved", oracle.BC_VIRTUAL_AVG, (3.0, 3.0), (1.2, 0.8), (0, 0), oracle.PAIR_CROSS),
    ("improved_self", oracle.BC_VIRTUAL_AVG, (2.0, 3.5), (0.7, 1.3), (0, 0), oracle.PAIR_SELF),
    ("constant", oracle.BC_CONSTANT, (3.0, 3.0), (1, 1), (0.3, 0.7), oracle.PAIR_CROSS),
]


def _random_state(nx, ny, mask, seed):
    rng = np.random.default_rng(seed)
    f = rng.uniform(0.001, 0.2, (2, 9, ny, nx))
    f *= (1 - mask)[None, None]
    return f


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("geom", ["periodic_salt", "walled_corner"])
def test_one_step_bruteforce(case, geom):
    _, bc, Gs, chi, rho_s, pairing = case
    tau = (0.9, 1.3)
    if geom == "periodic_salt":
        nx, ny = 7, 6
        mask = np.zeros((ny, nx), np.uint8)
        mask[1, 1] = 1       # isolated solid node
        mask[3, 3:6] = 1     # short wall segment
        mask[4, 5] = 1       # a corner
        ref_mask = mask
        periodic = True
        crop = (slice(None), slice(None))
    else:
        # 6x5 box with border walls and an interior corner; the reference
        # works on a copy padded with two solid layers (outside = solid)
        nx, ny = 6, 5
        mask = inputs.border_walls(nx, ny)
        mask[1, 3] = 1
        mask[2, 4] = 1
        ref_mask = np.pad(mask, 2, constant_values=1)
        periodic = False
        crop = (slice(2, 2 + ny), slice(2, 2 + nx))
    f = _random_state(nx, ny, mask, seed=7)
    o = oracle.Oracle(nx, ny, mask, tau=tau, G_AB=G, bc=bc, G_s=Gs, chi=chi, rho_s=rho_s,
                      pairing=pairing, periodic_x=periodic, periodic_y=periodic)
    o.f[...] = f
    rho, rt, F, u = o.fields()
    fpad = np.pad(f, ((0, 0), (0, 0), (2, 2), (2, 2))) if not periodic else f
    r_rho, r_rt, r_F, r_u, r_f = reference_step(fpad, ref_mask, bc, tau, Gs, chi, rho_s, pairing)
    c = (Ellipsis,) + crop
    np.testing.assert_allclose(rho, r_rho[c], rtol=0, atol=1e-14)
    np.testing.assert_allclose(rt, r_rt[c], rtol=0, atol=1e-14)
    np.testing.assert_allclose(F, r_F[c], rtol=0, atol=1e-14)
    np.testing.assert_allclose(u, r_u[c], rtol=0, atol=1e-14)
    o.step(1)
    np.testing.assert_allclose(o.f, r_f[c], rtol=0, atol=1e-14)
    # something non-trivial happened in every term
    assert np.abs(F).max() > 1e-3
    if bc == oracle.BC_VIRTUAL_AVG:
        assert np.count_nonzero(rt) > 0


def test_virtual_density_uniform_field():
    """On a uniform fluid the weighted mean of Eq. 8 is the fluid density, so
    rho~ = chi * rho exactly, whatever the wall shape."""
    nx, ny = 12, 10
    mask = inputs.border_walls(nx, ny)
    mask[4:6, 3:9] = 1
    mask[6, 7] = 1
    o = oracle.Oracle(nx, ny, mask, bc=oracle.BC_VIRTUAL_AVG, chi=(1.3, 0.6))
    o.init(np.full((ny, nx), 0.8), np.full((ny, nx), 0.25))
    rho, rt, F, u = o.fields()
    iface = o.interface_solid().astype(bool)
    assert iface.sum() > 10
    np.testing.assert_allclose(rt[0][iface], 1.3 * 0.8, rtol=1e-15)
    np.testing.assert_allclose(rt[1][iface], 0.6 * 0.25, rtol=1e-15)
    assert np.all(rt[:, ~iface] == 0)


def test_interface_solid_bruteforce():
    mask = inputs.random_solid_mask(16, 11, seed=3, fraction=0.35, periodic_x=True,
                                    periodic_y=False)
    o = oracle.Oracle(16, 11, mask, periodic_x=True)
    flag = o.interface_solid()
    ny, nx = mask.shape
    for y in range(ny):
        for x in range(nx):
            expect = 0
            if mask[y, x]:
                for dx in (-1, 0, 1):
                    for dy in (-1, 0, 1):
                        xx, yy = (x + dx) % nx, y + dy
                        if (dx or dy) and 0 <= yy < ny and mask[yy, xx] == 0:
                            expect = 1
            assert flag[y, x] == expect, (x, y)


def test_bounce_back_single_wall_node():
    """Halfway bounce-back at a flat wall: after one step with no force and
    tau = 1, a fluid node next to the wall receives, in each upward
    direction, its own post-collision population that pointed down."""
    nx, ny = 5, 5
    mask = inputs.border_walls(nx, ny, periodic_x=True)
    o = oracle.Oracle(nx, ny, mask, G_AB=0.0, periodic_x=True)
    rng = np.random.default_rng(1)
    o.f[...] = rng.uniform(0.01, 0.1, o.f.shape) * (1 - mask)
    rho, rt, F, u = o.fields()
    fpost = o.collide(rho, u, F)
    o.step(1)
    y = 1  # first fluid row
    for x in range(nx):
        # 2 (N) <- 4 (S), 5 (NE) <- 7 (SW), 6 (NW) <- 8 (SE)
        for i, j in ((2, 4), (5, 7), (6, 8)):
            assert o.f[0, i, y, x] == fpost[0, j, y, x]
            assert o.f[1, i, y, x] == fpost[1, j, y, x]


def test_reject_fluid_on_open_border():
    mask = np.zeros((5, 5), np.uint8)
    with pytest.raises(ValueError):
        oracle.Oracle(5, 5, mask)
    oracle.Oracle(5, 5, mask, periodic_x=True, periodic_y=True)
