"""Pins of the oracle against invariants and symmetries that the method
fixes: conservation of each component's mass under bounce-back, total
momentum with pairwise Shan-Chen forces, uniform states, mirror symmetries,
the A<->B exchange symmetry and the rest state on an on-grid wall."""
import numpy as np
import pytest

import oracle
from paper_2009_12584_gb300 import inputs

BCS = [
    ("mc", dict(bc=oracle.BC_MARTYS_CHEN, G_s=(-0.2, 0.2))),
    ("llkc", dict(bc=oracle.BC_LLKC, G_s=(-0.5, 0.5))),
    ("improved", dict(bc=oracle.BC_VIRTUAL_AVG, G_s=(3.0, 3.0), chi=(1.2, 0.8))),
    ("constant", dict(bc=oracle.BC_CONSTANT, G_s=(3.0, 3.0), rho_s=(0.4, 0.6))),
]


def momentum(o):
    rho, rt, F, u = o.fields()
    cx, cy, w, _ = oracle.lattice()
    jx = np.einsum("sixy,i->", o.f, cx.astype(float)) + 0.5 * F[:, 0].sum()
    jy = np.einsum("sixy,i->", o.f, cy.astype(float)) + 0.5 * F[:, 1].sum()
    return jx, jy, F


@pytest.mark.parametrize("name,kw", BCS, ids=[b[0] for b in BCS])
def test_mass_conserved_with_bounce_back(name, kw):
    nx, ny = 40, 30
    mask = inputs.inclined_wall_mask(nx, ny, 20.0, 7)
    rA, rB = inputs.sharp_droplet(nx, ny, nx / 2, ny / 2, 7)
    o = oracle.Oracle(nx, ny, mask, **kw).init(rA, rB)
    m0 = o.mass()
    o.step(300)
    m1 = o.mass()
    assert np.all(np.abs(m1 - m0) / m0 < 1e-12), (m0, m1)
    assert np.isfinite(o.f).all()


def test_uniform_state_is_stationary():
    nx, ny = 9, 7
    mask = np.zeros((ny, nx), np.uint8)
    o = oracle.Oracle(nx, ny, mask, periodic_x=True, periodic_y=True, tau=(0.8, 1.7))
    o.init(np.full((ny, nx), 0.7), np.full((ny, nx), 0.3))
    f0 = o.f.copy()
    rho, rt, F, u = o.fields()
    assert np.abs(F).max() == 0.0
    o.step(50)
    assert np.abs(o.f - f0).max() < 1e-15


def test_total_momentum_conserved_periodic():
    """Shan-Chen forces are pairwise antisymmetric, so in a periodic box with
    no solid their sum vanishes and the total momentum sum f c + F/2 is
    conserved (equal relaxation times)."""
    nx, ny = 16, 12
    mask = np.zeros((ny, nx), np.uint8)
    rA, rB, ux, uy = inputs.random_fields(nx, ny, seed=5, umax=0.02)
    o = oracle.Oracle(nx, ny, mask, periodic_x=True, periodic_y=True, tau=(1.1, 1.1))
    o.init(rA, rB, ux, uy)
    jx0, jy0, F = momentum(o)
    assert abs(F[:, 0].sum()) < 1e-13 and abs(F[:, 1].sum()) < 1e-13
    assert np.abs(F).max() > 1e-2
    o.step(100)
    jx1, jy1, _ = momentum(o)
    assert abs(jx1 - jx0) < 1e-12 and abs(jy1 - jy0) < 1e-12


@pytest.mark.parametrize("name,kw", BCS, ids=[b[0] for b in BCS])
def test_x_mirror_symmetry(name, kw):
    """A geometry and state symmetric under x -> nx-1-x stay symmetric."""
    nx, ny = 24, 16
    mask = inputs.border_walls(nx, ny)
    mask[1:3, :] = 1
    mask[3, 6:18] = 1          # a step on the floor
    rA, rB = inputs.sharp_droplet(nx, ny, (nx - 1) / 2, 5, 5)
    o = oracle.Oracle(nx, ny, mask, **kw).init(rA, rB)
    o.step(150)
    rho, rt, F, u = o.fields()
    np.testing.assert_allclose(rho, rho[:, :, ::-1], rtol=0, atol=1e-12)
    np.testing.assert_allclose(u[0], -u[0][:, ::-1], rtol=0, atol=1e-13)
    np.testing.assert_allclose(u[1], u[1][:, ::-1], rtol=0, atol=1e-13)
    assert np.abs(u).max() > 1e-4


@pytest.mark.parametrize("name,kw", BCS, ids=[b[0] for b in BCS])
def test_diagonal_symmetry(name, kw):
    """A square geometry and state symmetric under x <-> y stay symmetric: the
    x and y directions are treated alike."""
    n = 18
    mask = inputs.border_walls(n, n)
    mask[:4, :4] = 1
    mask[6, 9] = 1
    mask[9, 6] = 1
    rA, rB = inputs.sharp_droplet(n, n, 8, 8, 4)
    o = oracle.Oracle(n, n, mask, **kw).init(rA, rB)
    o.step(100)
    rho, rt, F, u = o.fields()
    np.testing.assert_allclose(rho, rho.transpose(0, 2, 1), rtol=0, atol=1e-12)
    np.testing.assert_allclose(u[0], u[1].T, rtol=0, atol=1e-13)


@pytest.mark.parametrize("kw", [
    dict(bc=oracle.BC_MARTYS_CHEN, G_s=(0.3, 0.3)),
    dict(bc=oracle.BC_LLKC, G_s=(-0.4, -0.4)),
    dict(bc=oracle.BC_VIRTUAL_AVG, G_s=(3.0, 3.0), chi=(1.3, 1.3)),
    dict(bc=oracle.BC_CONSTANT, G_s=(2.0, 2.0), rho_s=(0.5, 0.5)),
], ids=["mc", "llkc", "improved", "constant"])
def test_component_exchange_symmetry(kw):
    """With component-symmetric parameters, swapping A and B together with an
    x-mirror maps the dynamics onto itself: rho^A(x) = rho^B(mirror x)."""
    nx, ny = 20, 12
    mask = inputs.border_walls(nx, ny)
    x = np.arange(nx)[None, :]
    rA = np.where(x < nx / 2, 0.95, 0.06) * np.ones((ny, 1))
    rB = rA[:, ::-1].copy()
    o = oracle.Oracle(nx, ny, mask, **kw).init(rA, rB)
    o.step(120)
    rho, rt, F, u = o.fields()
    np.testing.assert_allclose(rho[0], rho[1][:, ::-1], rtol=0, atol=1e-12)


def test_droplet_on_grid_wall_stays_at_rest():
    """A droplet centred between two nodes on a wall aligned with the lattice
    (periodic along it) is mirror-symmetric about its centre, so its net
    tangential momentum is zero at all times: it does not slide."""
    nx, ny = 40, 24
    mask = inputs.flat_wall_mask(nx, ny)
    rA, rB = inputs.sharp_droplet(nx, ny, 17.5, 0.5, 9, 1.0, 0.03)
    for kw in (dict(bc=oracle.BC_MARTYS_CHEN, G_s=(-0.2, 0.2)),
               dict(bc=oracle.BC_VIRTUAL_AVG, G_s=(3.0, 3.0), chi=(1.1, 0.9))):
        o = oracle.Oracle(nx, ny, mask, periodic_x=True, **kw).init(rA, rB)
        for _ in range(4):
            o.step(50)
            jx, jy, _ = momentum(o)
            assert abs(jx) < 1e-12
