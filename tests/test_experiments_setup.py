"""Set-up of the paper-scale experiments (no GPU): the parameters the paper
prints follow from the stated relations (Sec. 4: Oh = 0.286, nu = 0.16 at
R0 = 12.5 in 175 x 125, nu = 0.92 at R0 = 400 in 5600 x 4000, tau = 1.88 for
nu = 0.46), the plane of Sec. 3.1 is tangent to the initial droplet, and the
slope fit recovers a known power law."""
import math

import numpy as np
import pytest

from paper_2009_12584_gb300 import experiments as ex


@pytest.mark.parametrize("R0,nx,ny,nu", [(12.5, 175, 125, 0.16), (100.0, 1400, 1000, 0.46),
                                         (400.0, 5600, 4000, 0.92)])
def test_coalescence_setup_matches_printed_parameters(R0, nx, ny, nu):
    s = ex.coalescence_setup(R0)
    assert (s["nx"], s["ny"]) == (nx, ny)
    assert abs(s["nu"] - nu) < 0.005  # the paper prints two decimals
    assert abs(s["nu"] / math.sqrt(ex.SIGMA * R0) - ex.OH) < 1e-12
    assert abs(s["tau_visc"] - s["nu"] * R0 / ex.SIGMA) < 1e-9
    xb, y0 = s["bridge"]
    assert xb == nx // 2 and s["mask"][y0 - 1, xb] == 1 and s["mask"][y0, xb] == 0
    assert (s["rhoA"] * s["mask"]).sum() == 0


def test_curved_surface_bridge_row_is_above_the_disk():
    s = ex.coalescence_setup(50.0, Rs=100.0)
    xb, y0 = s["bridge"]
    assert y0 >= s["ny"] // 2 and s["mask"][y0 - 1, xb] == 1 and s["mask"][y0, xb] == 0


def test_tau_of_nu():
    assert abs(ex.tau_from_nu(0.46) - 1.88) < 1e-12


@pytest.mark.parametrize("beta", [10.0, 20.0, 30.0, 45.0])
def test_wall_line_tangent_to_initial_droplet(beta):
    n, R0 = 1000, 100.0
    (x0, y0), ang = ex.wall_line(n, beta, R0)
    b = math.radians(ang)
    # distance from the droplet centre (n/2, n/2) to the line through (x0, y0) at angle b
    d = -(n / 2 - x0) * math.sin(b) + (n / 2 - y0) * math.cos(b)
    assert abs(d - R0) < 1e-9


def test_viscous_slope_recovers_power_law():
    t = np.arange(1, 400, dtype=float)
    b = 30.0 * (t / 200.0) ** 0.857
    assert abs(ex.viscous_slope(t, b, 60.0, 200.0) - 0.857) < 1e-10
    assert ex.viscous_slope(t[:2], b[:2], 60.0, 200.0) is None
    # an initial relaxation (overlapping smoothed interfaces) is left out
    b2 = b.copy()
    b2[:20] = np.linspace(12.0, 1.5 * b[20], 20)
    assert abs(ex.viscous_slope(t, b2, 60.0, 200.0) - 0.857) < 1e-10


def test_chi_mapping():
    assert ex.chi_from_xi(-0.2) == (1.2, 0.8)
