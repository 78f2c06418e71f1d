"""Parity of the on-device diagnostics (lbm_diagnostics) with the oracle's
measurement functions applied to the oracle's fields after the same steps.

FP64 storage: the fields agree to rounding (1e-12), so every crossing is
the same and the fits agree to ~1e-9. FP32 storage: densities differ by
~1e-6 after a few hundred steps, which moves each crossing by ~1e-5 and may
flip a crossing whose density sits within 1e-6 of the level; the bounds
below allow two such flips (one fitted point of a hundred moves the angle
by ~0.01 degree)."""
import math

import numpy as np
import pytest

import oracle
from oracle import diag as odiag
from paper_2009_12584_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2009_12584_gb300 import lbm  # noqa: E402


def _runs(nx, ny, mask, rA, rB, steps, okw, gkind, gkw, storage, periodic=(False, False)):
    o = oracle.Oracle(nx, ny, mask, periodic_x=periodic[0], periodic_y=periodic[1], **okw)
    o.init(rA, rB).step(steps)
    sim = lbm.Simulation(nx, ny, periodic_x=periodic[0], periodic_y=periodic[1], storage=storage)
    sim.set_geometry(mask).set_wetting(gkind, **gkw).init_fields(rA, rB).step(steps)
    rho, _, _, u = o.fields()
    return rho, u, sim


def _compare(rho, u, mask, sim, kw, fp64):
    d = sim.diagnostics(**kw)
    W, com, vel = odiag.weighted_com(rho[0], u, mask, kw["rho_out"])
    rel = 1e-11 if fp64 else 2e-5
    assert d["weight"] == pytest.approx(W, rel=rel)
    assert d["com"][0] == pytest.approx(com[0], rel=rel) and d["com"][1] == pytest.approx(com[1], rel=rel)
    vabs = 1e-13 if fp64 else 2e-7
    assert abs(d["com_velocity"][0] - vel[0]) < vabs and abs(d["com_velocity"][1] - vel[1]) < vabs
    t = kw["tangent"]
    assert abs(d["sliding_velocity"] - (vel[0] * t[0] + vel[1] * t[1])) < vabs
    assert abs(d["max_u"] - odiag.max_speed(u, mask)) < (1e-13 if fp64 else 2e-7)
    th, (xc, yc, R), n = odiag.contact_angle(rho[0], mask, kw["wall_point"], kw["wall_angle_deg"],
                                              kw["exclude"], kw["level"], kw.get("box"))
    if fp64:
        assert d["contour_points"] == n
        assert abs(d["contact_angle_deg"] - th) < 1e-7
        assert abs(d["circle"][0] - xc) < 1e-8 and abs(d["circle"][1] - yc) < 1e-8 and abs(d["circle"][2] - R) < 1e-8
    else:
        assert abs(d["contour_points"] - n) <= 2
        assert abs(d["contact_angle_deg"] - th) < 0.05
        assert abs(d["circle"][2] - R) < 0.05
    if kw.get("bridge") is not None:
        b = odiag.bridge_radius(rho[0], kw["bridge"][0], kw["bridge"][1], kw["level"])
        assert abs(d["bridge_radius"] - b) < (1e-10 if fp64 else 1e-3)
    return d


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_diag_sessile_flat_wall(storage):
    nx, ny = 120, 60
    mask = inputs.flat_wall_mask(nx, ny)
    rA, rB = inputs.sharp_droplet(nx, ny, nx / 2, 0.5, 18)
    rho, u, sim = _runs(nx, ny, mask, rA, rB, 300, dict(bc=oracle.BC_MARTYS_CHEN, G_s=(-0.2, 0.2)),
                        "martys_chen", dict(G_s=(-0.2, 0.2)), storage, periodic=(True, False))
    kw = dict(level=0.5, rho_out=0.055, tangent=(1.0, 0.0), wall_point=(0.0, 0.5), wall_angle_deg=0.0,
              exclude=3.0, bridge=(nx // 2, 1))
    d = _compare(rho, u, mask, sim, kw, storage == "fp64")
    assert 30.0 < d["contact_angle_deg"] < 90.0  # G_w < 0 wets the A phase
    assert d["bridge_radius"] > 10.0


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_diag_inclined_wall_improved(storage):
    nx, ny, beta, R0 = 150, 90, 20.0, 18
    mask = inputs.inclined_wall_mask(nx, ny, beta, R0)
    rA, rB = inputs.sharp_droplet(nx, ny, nx / 2, ny / 2, R0)
    rho, u, sim = _runs(nx, ny, mask, rA, rB, 250,
                        dict(bc=oracle.BC_VIRTUAL_AVG, G_s=(3.0, 3.0), chi=(0.8, 1.2)),
                        "virtual_avg", dict(G_s=(3.0, 3.0), chi=(0.8, 1.2)), storage)
    b = math.radians(beta)
    # a point of the wall line tangent to the initial droplet
    wp = (nx / 2 + R0 * math.sin(b), ny / 2 - R0 * math.cos(b))
    kw = dict(level=0.5, rho_out=0.055, tangent=(math.cos(b), math.sin(b)), wall_point=wp, wall_angle_deg=beta,
              exclude=3.0)
    _compare(rho, u, mask, sim, kw, storage == "fp64")


def test_diag_bridge_and_box_fp64():
    # two droplets on a flat wall whose feet touch: the bridge column is the
    # symmetry line; the box keeps the left droplet's contour only
    nx, ny = 140, 50
    mask = inputs.flat_wall_mask(nx, ny)
    rA1, rB1 = inputs.sharp_droplet(nx, ny, nx / 2 - 16, 0.5, 15)
    rA2, _ = inputs.sharp_droplet(nx, ny, nx / 2 + 16, 0.5, 15)
    rA = np.maximum(rA1, rA2)
    rB = np.where(rA > 0.5, rB1.min(), rB1.max())
    rho, u, sim = _runs(nx, ny, mask, rA, rB, 200, dict(bc=oracle.BC_LLKC, G_s=(-0.4, 0.4)),
                        "llkc", dict(G_s=(-0.4, 0.4)), "fp64", periodic=(True, False))
    kw = dict(level=0.5, rho_out=0.055, tangent=(1.0, 0.0), wall_point=(0.0, 0.5), wall_angle_deg=0.0,
              exclude=3.0, box=(0.0, nx / 2 - 1.0, 0.0, float(ny)), bridge=(nx // 2, 1))
    d = _compare(rho, u, mask, sim, kw, True)
    assert d["contour_points"] > 10


def test_diag_deterministic_and_errors():
    nx, ny = 64, 40
    mask = inputs.flat_wall_mask(nx, ny)
    rA, rB = inputs.sharp_droplet(nx, ny, nx / 2, 0.5, 12)
    sim = lbm.Simulation(nx, ny, periodic_x=True, storage="fp32")
    sim.set_geometry(mask).set_wetting("martys_chen", G_s=(-0.2, 0.2)).init_fields(rA, rB).step(50)
    a, b = sim.diagnostics(), sim.diagnostics()
    assert a == b
    with pytest.raises(lbm.LbmError):
        sim.diagnostics(level=2.5)
    with pytest.raises(lbm.LbmError):
        sim.diagnostics(bridge=(nx, 1))
    with pytest.raises(lbm.LbmError):
        sim.diagnostics(wall_point=(float("nan"), 0.5))
    # no contour inside an empty box: no circle
    d = sim.diagnostics(box=(1000.0, 1001.0, 0.0, 1.0))
    assert d["contour_points"] == 0 and math.isnan(d["contact_angle_deg"])


def test_diag_counts_nonfinite_nodes():
    # a diverged run, made on the host: one fluid node's populations set to NaN
    nx, ny = 64, 40
    mask = inputs.flat_wall_mask(nx, ny)
    rA, rB = inputs.sharp_droplet(nx, ny, nx / 2, 0.5, 12)
    sim = lbm.Simulation(nx, ny, periodic_x=True, storage="fp32")
    sim.set_geometry(mask).set_wetting("martys_chen", G_s=(-0.2, 0.2)).init_fields(rA, rB).step(20)
    d0 = sim.diagnostics()
    assert d0["nonfinite_nodes"] == 0 and math.isfinite(d0["max_u"])
    f = sim.populations()
    f[:, :, 20, 10] = float("nan")
    sim.set_populations(f)
    d1 = sim.diagnostics()
    assert d1["nonfinite_nodes"] >= 1 and math.isnan(d1["max_u"])
    assert math.isfinite(d1["weight"])  # the other sums leave those nodes out
