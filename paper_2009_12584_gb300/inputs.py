"""Seeded synthetic inputs shaped like the paper's test problems.

Geometry masks (uint8, 1 = solid, shape [ny, nx], node (x, y) at [y, x]) and
initial density fields (float64). This module holds none of the method's
arithmetic: it only draws and rasterises the inputs that both the CUDA path
and the FP64 oracle are given.

Recipes (arXiv:2009.12584):
  * inclined plane, Sec. 3.1: walls on the box borders plus the half plane
    below y = tan(beta) [x - L_X/2 - R0 sin(beta)] + L_Y/2 - R0 cos(beta);
    a node is solid iff it lies strictly below that line (evaluated at
    integer node coordinates) or on a border row/column;
  * sharp droplet, Sec. 3.1: rho_in inside radius R0 of the centre, rho_out
    outside, the other component the reverse;
  * smooth droplets on a circular surface, Sec. 4: the tanh profile printed
    there, with argument (r^2 - R0^2) / delta^2;
  * porous medium (throughput workload): non-overlapping disks placed by
    random sequential addition with periodic wrap until the solid fraction
    is reached, then sharp droplets of the majority component in the pores.
"""
from __future__ import annotations

import math

import numpy as np


def border_walls(nx: int, ny: int, periodic_x: bool = False,
                 periodic_y: bool = False) -> np.ndarray:
    """Solid rows/columns on every non-periodic border."""
    m = np.zeros((ny, nx), np.uint8)
    if not periodic_x:
        m[:, 0] = 1
        m[:, -1] = 1
    if not periodic_y:
        m[0, :] = 1
        m[-1, :] = 1
    return m


def inclined_wall_mask(nx: int, ny: int, beta_deg: float, R0: float) -> np.ndarray:
    """Border walls plus the staircase of an inclined plane tangent to a
    droplet of radius R0 centred in the box (Sec. 3.1)."""
    m = border_walls(nx, ny)
    b = math.radians(beta_deg)
    x = np.arange(nx, dtype=np.float64)
    y_wall = math.tan(b) * (x - nx / 2 - R0 * math.sin(b)) + ny / 2 - R0 * math.cos(b)
    y = np.arange(ny, dtype=np.float64)[:, None]
    m[y < y_wall[None, :]] = 1
    return m


def flat_wall_mask(nx: int, ny: int, rows: int = 1, top_wall: bool = True) -> np.ndarray:
    """Periodic-in-x channel: ``rows`` solid rows at the bottom (the wall
    along y = 0) and one solid row at the top."""
    m = np.zeros((ny, nx), np.uint8)
    m[:rows, :] = 1
    if top_wall:
        m[-1, :] = 1
    return m


def circle_surface_mask(nx: int, ny: int, xc: float, yc: float, Rs: float,
                        periodic: bool = True) -> np.ndarray:
    """Solid disk of radius Rs centred at (xc, yc) (Sec. 4)."""
    m = border_walls(nx, ny, periodic, periodic)
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    m[(x - xc) ** 2 + (y - yc) ** 2 <= Rs * Rs] = 1
    return m


def sharp_droplet(nx: int, ny: int, xc: float, yc: float, R: float,
                  rho_in: float = 1.0, rho_out: float = 0.055):
    """(rhoA, rhoB): rho_in / rho_out inside / outside the disk for A, the
    reverse for B (Sec. 3.1)."""
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    inside = (x - xc) ** 2 + (y - yc) ** 2 <= R * R
    rA = np.where(inside, rho_in, rho_out)
    rB = np.where(inside, rho_out, rho_in)
    return np.ascontiguousarray(rA), np.ascontiguousarray(rB)


def tanh_droplets(nx: int, ny: int, centres, yc: float, R0: float,
                  rho1: float = 1.0, rho2: float = 0.055, delta: float = 8.0):
    """(rhoA, rhoB) for droplets with the smoothed interface of Sec. 4."""
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    rA = np.full((ny, nx), rho2)
    rB = np.full((ny, nx), rho1)
    for xc in centres:
        bump = 0.5 * (rho1 - rho2) * (1.0 - np.tanh(((x - xc) ** 2 + (y - yc) ** 2 - R0 * R0)
                                                    / (delta * delta)))
        rA = rA + bump
        rB = rB - bump
    return np.ascontiguousarray(rA), np.ascontiguousarray(rB)


def _disk_offsets(r: int):
    d = np.arange(-r, r + 1)
    dy, dx = np.meshgrid(d, d, indexing="ij")
    keep = dx * dx + dy * dy <= r * r
    return dy[keep], dx[keep]


def porous_disks(nx: int, ny: int, solid_fraction: float = 0.4, rmin: int = 8,
                 rmax: int = 40, gap: int = 1, seed: int = 1,
                 max_tries: int = 2_000_000) -> np.ndarray:
    """Fully periodic medium of non-overlapping solid disks (integer radius
    uniform in [rmin, rmax]) added by random sequential addition until the
    solid fraction is reached. Disks keep ``gap`` fluid nodes between them."""
    rng = np.random.default_rng(seed)
    m = np.zeros((ny, nx), np.uint8)
    target = solid_fraction * nx * ny
    solid = 0
    tries = 0
    cache = {}
    while solid < target and tries < max_tries:
        tries += 1
        r = int(rng.integers(rmin, rmax + 1))
        cx = int(rng.integers(0, nx))
        cy = int(rng.integers(0, ny))
        if r + gap not in cache:
            cache[r + gap] = _disk_offsets(r + gap)
        if r not in cache:
            cache[r] = _disk_offsets(r)
        oy, ox = cache[r + gap]
        if m[(cy + oy) % ny, (cx + ox) % nx].any():
            continue
        oy, ox = cache[r]
        m[(cy + oy) % ny, (cx + ox) % nx] = 1
        solid += oy.size
    return m


def pore_droplets(mask: np.ndarray, a_fraction: float = 0.3, rmin: int = 8,
                  rmax: int = 32, seed: int = 2, rho_in: float = 1.0,
                  rho_out: float = 0.055, max_tries: int = 1_000_000):
    """(rhoA, rhoB) on a fully periodic box: sharp disks of the majority A
    phase (radius uniform in [rmin, rmax], centred on fluid nodes, wrapped)
    until ``a_fraction`` of the fluid nodes are A-rich. Solid nodes get 0."""
    ny, nx = mask.shape
    rng = np.random.default_rng(seed)
    a = np.zeros((ny, nx), bool)
    fluid = mask == 0
    n_fluid = int(fluid.sum())
    n_a = 0
    tries = 0
    cache = {}
    while n_a < a_fraction * n_fluid and tries < max_tries:
        tries += 1
        r = int(rng.integers(rmin, rmax + 1))
        cx = int(rng.integers(0, nx))
        cy = int(rng.integers(0, ny))
        if not fluid[cy, cx]:
            continue
        if r not in cache:
            cache[r] = _disk_offsets(r)
        oy, ox = cache[r]
        yy, xx = (cy + oy) % ny, (cx + ox) % nx
        sel = fluid[yy, xx] & ~a[yy, xx]
        a[yy[sel], xx[sel]] = True
        n_a += int(sel.sum())
    rA = np.where(a, rho_in, rho_out)
    rB = np.where(a, rho_out, rho_in)
    rA[~fluid] = 0.0
    rB[~fluid] = 0.0
    return np.ascontiguousarray(rA), np.ascontiguousarray(rB)


def random_fields(nx: int, ny: int, seed: int, lo: float = 0.05, hi: float = 1.0,
                  umax: float = 0.0):
    """Uniform random densities (and optional velocities) for parity tests
    that exercise every term at once."""
    rng = np.random.default_rng(seed)
    rA = rng.uniform(lo, hi, (ny, nx))
    rB = rng.uniform(lo, hi, (ny, nx))
    if umax > 0:
        ux = rng.uniform(-umax, umax, (ny, nx))
        uy = rng.uniform(-umax, umax, (ny, nx))
        return rA, rB, ux, uy
    return rA, rB, None, None


def random_solid_mask(nx: int, ny: int, seed: int, fraction: float = 0.2,
                      periodic_x: bool = True, periodic_y: bool = True) -> np.ndarray:
    """Salt-and-pepper solid nodes (plus walls on non-periodic borders): the
    degenerate geometry with isolated solid nodes, corners and one-node gaps."""
    rng = np.random.default_rng(seed)
    m = (rng.random((ny, nx)) < fraction).astype(np.uint8)
    m |= border_walls(nx, ny, periodic_x, periodic_y)
    return m


# Approximate linear maps from a target contact angle (degrees) to the
# wetting parameter of each scheme, read off flat-wall oracle runs (droplet
# radius 12, G_AB = 3, densities 1 / 0.055): Martys-Chen and LLKC G_w (with
# G_As = -G_Bs = G_w), and the improved scheme's xi' with chi = (1 + xi',
# 1 - xi'). They only spread the synthetic batch over wetting regimes.
def wetting_for_angle(bc: str, theta_deg: float):
    d = theta_deg - 90.0
    if bc == "martys_chen":
        gw = d / 135.0
        return dict(G_s=(gw, -gw))
    if bc == "llkc":
        gw = d / 37.0
        return dict(G_s=(gw, -gw))
    xi = -d / 112.0
    return dict(G_s=(3.0, 3.0), chi=(1.0 + xi, 1.0 - xi))


def batched_workload(n: int = 512, seed: int = 0, size_scale: float = 1.0):
    """Independent inclined-wall simulations: grid sizes uniform from 64x64
    to 512x256 (times size_scale), wall angle uniform in [0, 45] degrees,
    contact angle uniform in [45, 135] degrees, scheme uniform over
    Martys-Chen, LLKC and the improved virtual density; droplet radius
    min(nx, ny) / 6, sharp, tangent to the wall."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nx = int(rng.integers(64, 513) * size_scale)
        ny = int(rng.integers(64, 257) * size_scale)
        nx, ny = max(nx, 16), max(ny, 16)
        beta = float(rng.uniform(0.0, 45.0))
        theta = float(rng.uniform(45.0, 135.0))
        bc = ("martys_chen", "llkc", "virtual_avg")[int(rng.integers(0, 3))]
        R0 = min(nx, ny) / 6.0
        mask = inclined_wall_mask(nx, ny, beta, R0)
        rA, rB = sharp_droplet(nx, ny, nx / 2, ny / 2, R0)
        out.append(dict(nx=nx, ny=ny, beta=beta, theta=theta, bc=bc, wetting=wetting_for_angle(bc, theta),
                        mask=mask, rhoA=rA, rhoB=rB))
    return out
