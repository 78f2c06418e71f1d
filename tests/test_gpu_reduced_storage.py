"""Reduced-precision storage against the FP64 oracle at the bounds the
method is held to: the droplet's sliding velocity within 1e-6 (lattice
units) at every sample and its contact angle within 0.5 deg of the
oracle's, on the inclined-plane set-up of Sec. 3.1 at 400 x 200 with
R0 = 30 (walls on the borders, the plane tangent to the droplet), for the
three wetting schemes of Sec. 2 on a grid-aligned and a 20 deg plane,
10,000 steps.

The oracle's values are in tests/golden/oracle_accuracy.json, written by
tests/golden/make_oracle_accuracy.py from the oracle alone (the runs take
minutes on the host; test_oracle_accuracy_golden re-derives one sample).
The GPU side measures through lbm_diagnostics with the same definitions
(weight max(rho^A - 0.055, 0), Kasa fit of the rho^A = 0.5 crossings more
than 3 nodes from the plane's line and inside the same box).

FP32 storage and the 16-bit encodings with velocity references
(velocity_refs: deviations from w_i rho (1 + 3 c_i . u) of the writer)
must meet both bounds. The default 16-bit encodings (deviations from
w_i rho of the writer) must meet the contact-angle bound; they do not hold
the sliding velocity within 1e-6 over 10,000 steps in every case (the
16-bit rounding of the deviations changes the droplet's motion by parts in
1e4 to 1e3): where they miss, the case is marked xfail with the measured
error, which the design notes tabulate.
"""
import json
import math
import os

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2009_12584_gb300 import inputs, lbm  # noqa: E402

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_accuracy.json")))
BOUND_UD = 1e-6     # sliding velocity, lattice units
BOUND_THETA = 0.5   # contact angle, degrees
WETTING = {"mc": ("martys_chen", dict(G_s=(-0.2, 0.2))), "llkc": ("llkc", dict(G_s=(-0.5, 0.5))),
           "improved": ("virtual_avg", dict(G_s=(3.0, 3.0), chi=(1.2, 0.8)))}
# (storage, velocity_refs)
STORAGES = {"fp32": ("fp32", False), "fp16": ("fp16", False), "fp16u": ("fp16", True), "bf16": ("bf16", False),
            "bf16u": ("bf16", True)}


def _angle_defined(c):
    # Martys-Chen and LLKC droplets slide along the inclined plane until they
    # reach the box (Sec. 3.1); their fitted circle is then no contact angle
    return c["beta"] == 0.0 or c["scheme"] == "improved"


@pytest.mark.parametrize("storage", list(STORAGES))
@pytest.mark.parametrize("idx", range(len(GOLD["cases"])),
                         ids=[f"{c['scheme']}-beta{int(c['beta'])}" for c in GOLD["cases"]])
def test_sliding_velocity_and_contact_angle_vs_oracle(storage, idx):
    c = GOLD["cases"][idx]
    nx, ny, R0 = GOLD["nx"], GOLD["ny"], GOLD["R0"]
    b = math.radians(c["beta"])
    wp = (nx / 2 + R0 * math.sin(b), ny / 2 - R0 * math.cos(b))
    tvec = (math.cos(b), math.sin(b))
    mask = inputs.inclined_wall_mask(nx, ny, c["beta"], R0)
    rA, rB = inputs.sharp_droplet(nx, ny, nx / 2, ny / 2, R0)
    kind, wkw = WETTING[c["scheme"]]
    st, vref = STORAGES[storage]
    sim = lbm.Simulation(nx, ny, storage=st, velocity_refs=vref)
    sim.set_geometry(mask).set_wetting(kind, **wkw).init_fields(rA, rB)
    dkw = dict(level=GOLD["level"], rho_out=GOLD["rho_out"], tangent=tvec, wall_point=wp,
               wall_angle_deg=c["beta"], exclude=GOLD["exclude"], box=tuple(GOLD["box"]))
    worst = 0.0
    for ud_oracle in c["sliding_velocity"]:
        sim.step(c["every"])
        d = sim.diagnostics(**dkw)
        worst = max(worst, abs(d["sliding_velocity"] - ud_oracle))
    if _angle_defined(c):
        assert abs(d["contact_angle_deg"] - c["contact_angle_deg"]) <= BOUND_THETA, \
            (d["contact_angle_deg"], c["contact_angle_deg"])
    sim.close()
    if storage == "fp32" or vref:
        assert worst <= BOUND_UD, (storage, worst)
    elif worst > BOUND_UD:
        pytest.xfail(f"{storage}: sliding velocity off by {worst:.2e} (bound {BOUND_UD:.0e})")
