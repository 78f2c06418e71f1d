"""Write oracle_experiments.json: the FP64 oracle's measurements on reduced
forms of the paper's two parametric studies, to which the library's
experiment drivers are held.

  - contact-angle sweep (Sec. 3.2): a sharp droplet of radius R0 = 20 on
    the staircase plane of Sec. 3.1 in a 160 x 160 box (walls on the
    borders, the plane tangent to the droplet), improved virtual-density
    scheme with the D2Q25 average of Eq. 8, G_sigma_s = G_AB = 3,
    tau = 1.88, xi in {-0.2, +0.2} mapped to chi = (1 - xi, 1 + xi) (Eq. 7
    as printed), beta in {0, 10, 20} deg; every ``check`` steps: the
    contact angle (Kasa circle through the rho^A = 0.5 crossings more than
    3 nodes from the plane's line; on a grid-aligned plane the line is the
    halfway plane above the last solid row), the sliding velocity along the
    plane (weight max(rho^A - 0.055, 0)) and max |u|;
  - coalescence (Sec. 4): two droplets with the printed tanh profile
    (delta = 8, densities 1 / 0.055) of radius R0 = 25 on a flat wall in
    a 14 R0 x 10 R0 box periodic in x, centred R0 sin(theta_c) + 1 either
    side of the middle at height L_Y / 2 - R0 cos(theta_c), theta_c = 71 deg
    (xi = -0.2), viscosity nu = Oh sqrt(sigma R0) with Oh = 0.286 and
    sigma = 0.026, up to t = tau_nu = nu R0 / sigma; the bridge radius on
    the middle column (from the halfway wall to the rho^A = 0.5 crossing)
    every ``every`` steps.

Only the oracle and the seeded input recipes are used here.

    python tests/golden/make_oracle_experiments.py
"""
import json
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle import diag  # noqa: E402
from paper_2009_12584_gb300 import inputs  # noqa: E402

RHO_OUT = 0.055
SWEEP = dict(n=160, R0=20.0, tau=1.88, xis=[-0.2, 0.2], betas=[0.0, 10.0, 20.0], steps=9000, check=3000)
COAL = dict(R0=25.0, theta_c=71.0, xi=-0.2, Oh=0.286, sigma=0.026, delta=8.0, samples=20)


def sweep_case(xi, beta):
    n, R0 = SWEEP["n"], SWEEP["R0"]
    mask = inputs.inclined_wall_mask(n, n, beta, R0)
    rA, rB = inputs.sharp_droplet(n, n, n / 2, n / 2, R0)
    tau = SWEEP["tau"]
    o = oracle.Oracle(n, n, mask, tau=(tau, tau), bc=oracle.BC_VIRTUAL_AVG, G_s=(3.0, 3.0),
                      chi=(1.0 - xi, 1.0 + xi), avg_stencil=25).init(rA, rB)
    b = math.radians(beta)
    wp = (n / 2 + R0 * math.sin(b), n / 2 - R0 * math.cos(b))
    if beta == 0.0:
        wp = (wp[0], math.ceil(wp[1]) - 0.5)
    checks = []
    for t in range(SWEEP["check"], SWEEP["steps"] + 1, SWEEP["check"]):
        o.step(SWEEP["check"])
        rho, _, _, u = o.fields()
        th, circle, npts = diag.contact_angle(rho[0], mask, wp, beta)
        checks.append(dict(step=t, theta_deg=th, contour_points=npts,
                           sliding_velocity=diag.sliding_velocity(rho[0], u, mask, RHO_OUT,
                                                                  (math.cos(b), math.sin(b))),
                           max_u=diag.max_speed(u, mask)))
    return dict(xi=xi, beta=beta, checks=checks)


def coalescence_case():
    R0 = COAL["R0"]
    nx, ny = int(round(14 * R0)), int(round(10 * R0))
    mask = inputs.flat_wall_mask(nx, ny, rows=ny // 2)
    th = math.radians(COAL["theta_c"])
    dx = R0 * math.sin(th) + 1.0
    rA, rB = inputs.tanh_droplets(nx, ny, (nx / 2 - dx, nx / 2 + dx), ny / 2 - R0 * math.cos(th), R0, 1.0,
                                  RHO_OUT, COAL["delta"])
    rA, rB = rA * (1 - mask), rB * (1 - mask)
    nu = COAL["Oh"] * math.sqrt(COAL["sigma"] * R0)
    tau = 3.0 * nu + 0.5
    tau_visc = nu * R0 / COAL["sigma"]
    xi = COAL["xi"]
    o = oracle.Oracle(nx, ny, mask, tau=(tau, tau), bc=oracle.BC_VIRTUAL_AVG, G_s=(3.0, 3.0),
                      chi=(1.0 - xi, 1.0 + xi), periodic_x=True).init(rA, rB)
    xb = nx // 2
    y0 = next(y for y in range(1, ny - 1) if mask[y, xb] == 0 and mask[y - 1, xb] == 1)
    total = max(1, int(round(tau_visc)))
    every = max(1, total // COAL["samples"])
    ts, bs = [], []
    done = 0
    while done < total:
        k = min(every, total - done)
        o.step(k)
        done += k
        rho = o.fields()[0]
        ts.append(done)
        bs.append(diag.bridge_radius(rho[0], xb, y0))
    return dict(nx=nx, ny=ny, tau=tau, tau_visc=tau_visc, bridge=[xb, y0], steps=total, t=ts, b=bs)


def main():
    out = dict(sweep=dict(SWEEP, runs=[]), coalescence=dict(COAL))
    for beta in SWEEP["betas"]:
        for xi in SWEEP["xis"]:
            t0 = time.time()
            r = sweep_case(xi, beta)
            out["sweep"]["runs"].append(r)
            c = r["checks"][-1]
            print(f"sweep xi={xi} beta={beta}: theta={c['theta_deg']:.3f} u_d={c['sliding_velocity']:.3e} "
                  f"({time.time() - t0:.0f} s)", flush=True)
    t0 = time.time()
    out["coalescence"].update(coalescence_case())
    print(f"coalescence: b(end)={out['coalescence']['b'][-1]:.4f} after {out['coalescence']['steps']} steps "
          f"({time.time() - t0:.0f} s)", flush=True)
    with open(os.path.join(HERE, "oracle_experiments.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
