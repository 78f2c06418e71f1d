"""Pins of the oracle's lattice tables, equilibrium (Eq. 2) and Guo source
(Eq. 4) against values the paper prints and closed-form moment identities."""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_weights(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        r2, num, den, mult = (int(v) for v in line.split())
        rows.append((r2, Fraction(num, den), mult))
    return rows


def test_d2q9_weights_match_paper():
    cx, cy, w, opp = oracle.lattice()
    for r2, wt, mult in _read_weights("d2q9_weights.txt"):
        sel = (cx * cx + cy * cy) == r2
        assert sel.sum() == mult
        assert np.all(w[sel] == float(wt))


def test_d2q9_isotropy_and_opposites():
    cx, cy, w, opp = oracle.lattice()
    assert len(set(zip(cx.tolist(), cy.tolist()))) == 9
    assert abs(w.sum() - 1.0) < 1e-15
    assert abs((w * cx).sum()) < 1e-15 and abs((w * cy).sum()) < 1e-15
    # second moments: c_s^2 delta_ab with c_s^2 = 1/3
    assert abs((w * cx * cx).sum() - 1 / 3) < 1e-15
    assert abs((w * cy * cy).sum() - 1 / 3) < 1e-15
    assert abs((w * cx * cy).sum()) < 1e-15
    # fourth moments: c_s^4 (d_ab d_cd + d_ac d_bd + d_ad d_bc)
    assert abs((w * cx**4).sum() - 3 / 9) < 1e-15
    assert abs((w * cx**2 * cy**2).sum() - 1 / 9) < 1e-15
    for i in range(9):
        assert cx[opp[i]] == -cx[i] and cy[opp[i]] == -cy[i]


def test_d2q25_weights_match_paper():
    ex, ey, W = oracle.d2q25()
    assert len(set(zip(ex.tolist(), ey.tolist()))) == 24
    assert np.all(np.maximum(np.abs(ex), np.abs(ey)) <= 2)
    r2 = ex * ex + ey * ey
    for k, wt, mult in _read_weights("d2q25_weights.txt"):
        sel = r2 == k
        assert sel.sum() == mult
        assert np.all(W[sel] == float(wt))


def test_d2q25_moments():
    ex, ey, W = oracle.d2q25()
    # normalisation of the printed set: sum W c_x^2 = 1, odd moments vanish
    assert abs((W * ex * ex).sum() - 1.0) < 1e-15
    assert abs((W * ex).sum()) < 1e-15 and abs((W * ex * ey).sum()) < 1e-15
    # fourth-order isotropy: sum W c_x^4 = 3 sum W c_x^2 c_y^2
    assert abs((W * ex**4).sum() - 3 * (W * ex**2 * ey**2).sum()) < 1e-15
    # the weights do not sum to one (Eq. 8 divides by their fluid sum)
    assert abs(W.sum() - 173 / 140) < 1e-15


@pytest.mark.parametrize("seed", range(5))
def test_equilibrium_moments(seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.02, 1.2)
    ux, uy = rng.uniform(-0.1, 0.1, 2)
    cx, cy, w, _ = oracle.lattice()
    feq = oracle.equilibrium(rho, ux, uy)
    cs2 = 1 / 3
    assert abs(feq.sum() - rho) < 1e-15
    assert abs((feq * cx).sum() - rho * ux) < 1e-15
    assert abs((feq * cy).sum() - rho * uy) < 1e-15
    assert abs((feq * cx * cx).sum() - rho * (cs2 + ux * ux)) < 1e-15
    assert abs((feq * cy * cy).sum() - rho * (cs2 + uy * uy)) < 1e-15
    assert abs((feq * cx * cy).sum() - rho * ux * uy) < 1e-15
    # u = 0 reduces to rho * w_i
    assert np.allclose(oracle.equilibrium(rho, 0.0, 0.0), rho * w, rtol=0, atol=1e-16)


@pytest.mark.parametrize("seed", range(5))
def test_guo_source_moments(seed):
    rng = np.random.default_rng(100 + seed)
    tau = rng.uniform(0.6, 2.0)
    ux, uy = rng.uniform(-0.1, 0.1, 2)
    Fx, Fy = rng.uniform(-0.01, 0.01, 2)
    cx, cy, w, _ = oracle.lattice()
    S = oracle.source(tau, ux, uy, Fx, Fy)
    k = 1 - 1 / (2 * tau)
    assert abs(S.sum()) < 1e-16
    assert abs((S * cx).sum() - k * Fx) < 1e-16
    assert abs((S * cy).sum() - k * Fy) < 1e-16
    assert abs((S * cx * cx).sum() - k * 2 * ux * Fx) < 1e-16
    assert abs((S * cy * cy).sum() - k * 2 * uy * Fy) < 1e-16
    assert abs((S * cx * cy).sum() - k * (ux * Fy + uy * Fx)) < 1e-16
