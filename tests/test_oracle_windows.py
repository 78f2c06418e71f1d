"""The window method of the full-size parity test, checked with the oracle
alone: one step of a window cut with a margin of 5 nodes and closed by a
solid frame reproduces, in its interior, one step of the whole periodic
domain (the reach of one step is 4 nodes: populations 1, densities 2,
virtual densities of Eq. 8 4). A margin of 3 does not."""
import numpy as np
import pytest

import oracle
from paper_2009_12584_gb300 import inputs

N, W = 160, 24
CHI = (1.2, 0.8)


def _window_step_error(o_full, f_before, mask, x0, y0, M):
    span = W + 2 * M + 2
    pm = np.ascontiguousarray(mask[y0:y0 + span, x0:x0 + span]).copy()
    pm[0, :] = pm[-1, :] = 1
    pm[:, 0] = pm[:, -1] = 1
    o = oracle.Oracle(span, span, pm, bc=oracle.BC_VIRTUAL_AVG, G_s=(3.0, 3.0), chi=CHI)
    o.f[...] = f_before[:, :, y0:y0 + span, x0:x0 + span] * (pm == 0)[None, None]
    o.step(1)
    s = slice(M + 1, M + 1 + W)
    fluid = pm[s, s] == 0
    full = o_full.f[:, :, y0 + M + 1:y0 + M + 1 + W, x0 + M + 1:x0 + M + 1 + W]
    return np.abs(o.f[:, :, s, s] - full)[:, :, fluid].max()


@pytest.fixture(scope="module")
def domain():
    mask = inputs.porous_disks(N, N, solid_fraction=0.40, rmin=4, rmax=12, seed=3)
    rA, rB = inputs.pore_droplets(mask, a_fraction=0.35, rmin=3, rmax=10, seed=4)
    o = oracle.Oracle(N, N, mask, periodic_x=True, periodic_y=True, bc=oracle.BC_VIRTUAL_AVG, G_s=(3.0, 3.0),
                      chi=CHI).init(rA, rB).step(10)
    f_before = o.f.copy()
    o.step(1)
    return mask, f_before, o


@pytest.mark.parametrize("x0,y0", [(10, 20), (60, 70), (100, 30)])
def test_margin_five_is_exact(domain, x0, y0):
    mask, f_before, o = domain
    assert _window_step_error(o, f_before, mask, x0, y0, 5) < 1e-14


def test_margin_three_is_not(domain):
    mask, f_before, o = domain
    errs = [_window_step_error(o, f_before, mask, x0, y0, 3) for x0, y0 in [(10, 20), (60, 70), (100, 30)]]
    assert max(errs) > 1e-8
