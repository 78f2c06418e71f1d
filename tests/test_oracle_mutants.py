"""The pins catch plausible mistakes: copies of the oracle, each compiled
with one planted mistake (a dropped term, a wrong sign, index or weight, a
transposed operand), must fail at least one of the pin checks below, while
the unmodified source passes all of them."""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from paper_2009_12584_gb300 import inputs

SRC = os.path.join(os.path.dirname(oracle.__file__), "lbm_oracle.c")

MUTANTS = {
    "d2q25_weight": ("case 1: return 4.0 / 21.0;", "case 1: return 4.0 / 20.0;"),
    "eq8_solid_indicator": ("double fluid = 1.0 - phi(mask, m);", "double fluid = 1.0 - (1 - phi(mask, m));"),
    "guo_sign": ("- ux / CS2;", "+ ux / CS2;"),
    "sc_force_sign": ("fsc_x *= -rho[s * N + n] * p->G_AB;", "fsc_x *= rho[s * N + n] * p->G_AB;"),
    "adhesion_component": ("fs_x *= -rho[s * N + n] * p->G_s[s];", "fs_x *= -rho[s * N + n] * p->G_s[1 - s];"),
    "bounce_same_slot": ("v = fpost[(s * 9 + oi) * N + n];", "v = fpost[(s * 9 + i) * N + n];"),
    "half_force_dropped": ("jx += F[(s * 2 + 0) * N + n] / 2.0;", "jx += 0.0 * F[(s * 2 + 0) * N + n];"),
    "feq_u2_term": ("- u2 / (2.0 * CS2));", "- u2 / (2.0 * CS2 * CS2));"),
    "pairing_swapped": ("int cs = (p->pairing == ORACLE_PAIR_SELF) ? s : sb;",
                        "int cs = (p->pairing == ORACLE_PAIR_SELF) ? sb : s;"),
    "chi_index": ("rt[s * N + n] = p->chi[s] * num / den;", "rt[s * N + n] = p->chi[1 - s] * num / den;"),
    "cy_transposed": ("static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};",
                      "static const int CY[9] = {0, 0, 1, 0, -1, 1, -1, 1, -1};"),
    "sc_neighbour_component": ("fsc_x += W9[i] * rho[sb * N + m] * CX[i];",
                               "fsc_x += W9[i] * rho[s * N + m] * CX[i];"),
    "tau_ratio": ("fi - (fi - feq[i]) / p->tau[s] + S[i];", "fi - (fi - feq[i]) * p->tau[s] + S[i];"),
}


def build_variant(tmp, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site of {name} not found"
    path = os.path.join(tmp, f"{name}.c")
    open(path, "w").write(src.replace(old, new, 1))
    lib = os.path.join(tmp, f"lib{name}.so")
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-I", os.path.dirname(SRC), "-o", lib,
                           path, "-lm"])
    return oracle.load_library(lib)


def pins(lib):
    """A compact set of the pins of test_oracle_*: True when all hold."""
    from tests.test_oracle_bruteforce import CASES, reference_step
    cx, cy, w, opp = oracle.lattice(lib)
    ok = abs((w * cx * cx).sum() - 1 / 3) < 1e-15 and abs((w * cx * cy).sum()) < 1e-15
    ok &= all(cx[opp[i]] == -cx[i] and cy[opp[i]] == -cy[i] for i in range(9))
    ex, ey, W = oracle.d2q25(lib)
    ok &= abs((W * ex * ex).sum() - 1.0) < 1e-15
    feq = oracle.equilibrium(0.7, 0.03, -0.02, lib)
    ok &= abs((feq * cx * cx).sum() - 0.7 * (1 / 3 + 0.03 ** 2)) < 1e-15
    S = oracle.source(1.3, 0.03, -0.02, 0.01, 0.005, lib)
    ok &= abs(S.sum()) < 1e-16 and abs((S * cx).sum() - (1 - 0.5 / 1.3) * 0.01) < 1e-16
    # one step against the hand-expanded reference, every scheme
    nx, ny = 7, 6
    mask = np.zeros((ny, nx), np.uint8)
    mask[1, 1] = 1
    mask[3, 3:6] = 1
    mask[4, 5] = 1
    rng = np.random.default_rng(7)
    f = rng.uniform(0.001, 0.2, (2, 9, ny, nx)) * (1 - mask)[None, None]
    for _, bc, Gs, chi, rho_s, pairing in CASES:
        o = oracle.Oracle(nx, ny, mask, tau=(0.9, 1.3), G_AB=3.0, bc=bc, G_s=Gs, chi=chi, rho_s=rho_s,
                          pairing=pairing, periodic_x=True, periodic_y=True, lib=lib)
        o.f[...] = f
        r = reference_step(f, mask, bc, (0.9, 1.3), Gs, chi, rho_s, pairing)
        o.step(1)
        ok &= np.abs(o.f - r[4]).max() < 1e-14
    # mass with bounce-back
    nx, ny = 30, 20
    mask = inputs.inclined_wall_mask(nx, ny, 20.0, 5)
    rA, rB = inputs.sharp_droplet(nx, ny, nx / 2, ny / 2, 5)
    o = oracle.Oracle(nx, ny, mask, bc=oracle.BC_MARTYS_CHEN, G_s=(-0.2, 0.2), lib=lib).init(rA, rB)
    m0 = o.mass()
    o.step(50)
    ok &= bool(np.all(np.abs(o.mass() - m0) / m0 < 1e-12))
    return bool(ok)


def test_unmodified_oracle_passes_the_pins():
    assert pins(oracle._load())


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name):
    with tempfile.TemporaryDirectory() as tmp:
        lib = build_variant(tmp, name, *MUTANTS[name])
        assert not pins(lib), f"mutant {name} passed every pin"
