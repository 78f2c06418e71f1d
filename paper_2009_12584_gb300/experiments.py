"""Paper-scale experiments of arXiv:2009.12584 run through the library, with
every measurement taken on the device (``Simulation.diagnostics``):

- ``contact_angle_sweep`` (Sec. 3.2): a droplet on a plane inclined at beta
  under the improved virtual-density scheme, 1000 x 1000, tau = 1.88,
  R0 = 100; the equilibrium contact angle as a function of xi and beta (the
  paper reports the droplet at rest for every beta and theta = 71 degrees at
  xi = -0.2, quoted in Sec. 4). All runs of the sweep advance together as
  one batch.
- ``coalescence`` (Sec. 4): two droplets with contact angle theta_c on a
  flat (or circular) surface, smoothed initial interfaces, box 14 R0 x 10 R0;
  the bridge radius b(t) on the symmetry column, in the reduced units of the
  paper (t / tau_nu with tau_nu = eta R0 / sigma, b / R0), and the slope of
  log b against log t in the viscous regime.
- ``convergence``: ``coalescence`` on a flat surface at fixed Ohnesorge
  number Oh = nu / sqrt(sigma R0) = 0.286 for R0 = 12.5 ... 400 (175 x 125 up
  to 5600 x 4000), whose viscous slope the paper shows approaching the 2-D
  prediction 0.857.

Readings (shared with the rest of the library): xi maps to
chi = (1 - xi, 1 + xi) with Eq. 7 as printed; sigma = 0.026 is the value
the paper uses for Oh and tau_nu; nu = (tau - 1/2) / 3; the viscous window
of the slope fit is b / R0 in [0.05, 1/3] after the early minimum of b
(the paper puts the crossover at b ~ R0 / 3).

    python -m paper_2009_12584_gb300.experiments sweep [--n 1000 --steps 200000]
    python -m paper_2009_12584_gb300.experiments convergence [--radii 12.5 25 50 100 200 400]
    python -m paper_2009_12584_gb300.experiments slide     # inclined walls, FP32 vs FP64
    python -m paper_2009_12584_gb300.experiments curved    # coalescence on a disk, FP32/16 vs FP64
    python -m paper_2009_12584_gb300.experiments curvature # Fig. 8A: b(t) on disks of several radii
    python -m paper_2009_12584_gb300.experiments viscosity # Fig. 8B: b(t) at several viscosities
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time

import numpy as np

from . import inputs, lbm

SIGMA = 0.026       # surface tension the paper uses at G_AB = 3 (Sec. 4)
OH = 0.286          # Ohnesorge number of the convergence study (Sec. 4)
THETA_C = 71.0      # contact angle of the coalescence runs, xi = -0.2 (Sec. 4)
XI_C = -0.2


def chi_from_xi(xi: float):
    """chi^A, chi^B of Eq. 8 for the paper's xi (xi < 0 hydrophilic)."""
    return (1.0 - xi, 1.0 + xi)


def tau_from_nu(nu: float) -> float:
    return 3.0 * nu + 0.5


def wall_line(n: int, beta_deg: float, R0: float, ny=None):
    """A point of the staircase plane of Sec. 3.1 and its direction: the line
    y = tan(beta) (x - L_X/2 - R0 sin(beta)) + L_Y/2 - R0 cos(beta), tangent
    to the initial droplet (L_X = n, L_Y = ny or n). On a flat wall
    (beta = 0) the point is moved to the halfway plane above the last solid
    row."""
    b = math.radians(beta_deg)
    ly = n if ny is None else ny
    x0, y0 = n / 2 + R0 * math.sin(b), ly / 2 - R0 * math.cos(b)
    if beta_deg == 0.0:
        y0 = math.ceil(y0) - 0.5
    return (x0, y0), beta_deg


def contact_angle_sweep(xis=(-0.4, -0.2, 0.0, 0.2, 0.4), betas=(0.0, 10.0, 20.0, 30.0, 45.0), *, n=1000,
                        R0=100.0, tau=1.88, steps=200000, check_every=50000, avg_stencil=25, storage="fp32"):
    """Equilibrium contact angle (and sliding velocity, max |u|) of a
    droplet on the inclined plane for every (xi, beta), improved scheme.
    Returns the parameters and one record per run with every check."""
    runs = []
    for beta in betas:
        mask = inputs.inclined_wall_mask(n, n, beta, R0)
        rA, rB = inputs.sharp_droplet(n, n, n / 2, n / 2, R0)
        for xi in xis:
            sim = lbm.Simulation(n, n, tau=(tau, tau), storage=storage)
            sim.set_geometry(mask).set_wetting("virtual_avg", G_s=(3.0, 3.0), chi=chi_from_xi(xi),
                                               avg_stencil=avg_stencil)
            sim.init_fields(rA, rB)
            runs.append({"xi": xi, "beta": beta, "sim": sim, "checks": []})
    batch = lbm.Batch([r["sim"] for r in runs])
    done, t0 = 0, time.time()
    while done < steps:
        k = min(check_every, steps - done)
        batch.step(k)
        done += k
        for r in runs:
            wp, ang = wall_line(n, r["beta"], R0)
            b = math.radians(r["beta"])
            d = r["sim"].diagnostics(level=0.5, rho_out=0.055, tangent=(math.cos(b), math.sin(b)),
                                     wall_point=wp, wall_angle_deg=ang, exclude=3.0)
            r["checks"].append({"step": done, "theta_deg": d["contact_angle_deg"],
                                "sliding_velocity": d["sliding_velocity"], "max_u": d["max_u"],
                                "contour_points": d["contour_points"]})
    wall = time.time() - t0
    batch.close()
    out = []
    for r in runs:
        r["sim"].close()
        out.append({"xi": r["xi"], "beta": r["beta"], "checks": r["checks"]})
    return {"n": n, "R0": R0, "tau": tau, "steps": steps, "avg_stencil": avg_stencil, "storage": storage,
            "wall_s": wall, "runs": out}


def coalescence_setup(R0: float, *, Rs=None, theta_c=THETA_C, Oh=OH, sigma=SIGMA, delta=8.0, nu=None):
    """Grid, mask, initial densities and parameters of the Sec. 4 runs: box
    14 R0 x 10 R0; surface (x - L_X/2)^2 + (y - (L_Y/2 - Rs))^2 = Rs^2, or
    the half plane y < L_Y/2 for Rs = None; droplets centred at
    x = L_X/2 -+ (R0 sin(theta_c) + 1), y = L_Y/2 - R0 cos(theta_c) with the
    printed tanh profile; nu = Oh sqrt(sigma R0)."""
    nx, ny = int(round(14 * R0)), int(round(10 * R0))
    if Rs is None:
        mask = inputs.flat_wall_mask(nx, ny, rows=ny // 2)
    else:
        mask = inputs.circle_surface_mask(nx, ny, nx / 2, ny / 2 - Rs, Rs, periodic=True)
        mask[-1, :] = 1
        mask[0, :] = 1
    th = math.radians(theta_c)
    dx = R0 * math.sin(th) + 1.0
    rA, rB = inputs.tanh_droplets(nx, ny, (nx / 2 - dx, nx / 2 + dx), ny / 2 - R0 * math.cos(th), R0,
                                  1.0, 0.055, delta)
    rA, rB = rA * (1 - mask), rB * (1 - mask)
    if nu is None:
        nu = Oh * math.sqrt(sigma * R0)
    xb = nx // 2
    col = mask[:, xb]
    # first fluid node above the surface, whose top is at y = L_Y / 2
    y0 = next(y for y in range(max(1, ny // 2 - 2), ny - 1) if col[y] == 0 and col[y - 1] == 1)
    return {"nx": nx, "ny": ny, "mask": mask, "rhoA": rA, "rhoB": rB, "nu": nu, "tau": tau_from_nu(nu),
            "tau_visc": nu * R0 / sigma, "bridge": (xb, y0)}


def viscous_slope(t, b, R0, tau_visc, window=(0.05, 1.0 / 3.0)):
    """Least-squares slope of log(b/R0) against log(t/tau_visc) over the
    samples with b/R0 inside ``window`` that come after the smallest b seen
    before the window's upper end (smoothed initial interfaces that already
    overlap first relax); None with fewer than 3 samples."""
    t, b = np.asarray(t, float), np.asarray(b, float)
    inside = np.nonzero(b / R0 <= window[1])[0]
    if len(inside) == 0:
        return None
    i0 = int(np.argmin(b[: inside[-1] + 1]))
    sel = (b / R0 >= window[0]) & (b / R0 <= window[1]) & (t > 0) & (np.arange(len(t)) >= i0)
    if sel.sum() < 3:
        return None
    return float(np.polyfit(np.log(t[sel] / tau_visc), np.log(b[sel] / R0), 1)[0])


def coalescence(R0: float, *, Rs=None, t_end=1.0, samples=200, storage="fp32", xi=XI_C, theta_c=THETA_C,
                nu=None):
    """b(t) of two coalescing droplets up to t_end viscous times (nu: the
    kinematic viscosity, else the one of Oh = 0.286)."""
    s = coalescence_setup(R0, Rs=Rs, theta_c=theta_c, nu=nu)
    sim = lbm.Simulation(s["nx"], s["ny"], tau=(s["tau"], s["tau"]), periodic_x=True, storage=storage)
    sim.set_geometry(s["mask"]).set_wetting("virtual_avg", G_s=(3.0, 3.0), chi=chi_from_xi(xi))
    sim.init_fields(s["rhoA"], s["rhoB"])
    total = max(1, int(round(t_end * s["tau_visc"])))
    every = max(1, total // samples)
    ts, bs, us = [], [], []
    t0 = time.time()
    done = 0
    while done < total:
        k = min(every, total - done)
        sim.step(k)
        done += k
        d = sim.diagnostics(bridge=s["bridge"], wall_point=(0.0, s["bridge"][1] - 0.5))
        ts.append(done)
        bs.append(d["bridge_radius"])
        us.append(d["max_u"])
    wall = time.time() - t0
    sim.close()
    return {"R0": R0, "Rs": Rs, "nx": s["nx"], "ny": s["ny"], "nu": s["nu"], "tau": s["tau"],
            "tau_visc": s["tau_visc"], "steps": total, "wall_s": wall, "t": ts, "b": bs, "max_u": us,
            "slope": viscous_slope(ts, bs, R0, s["tau_visc"])}


def convergence(radii=(12.5, 25.0, 50.0, 100.0, 200.0, 400.0), *, t_end=1.0, storage="fp32"):
    return [coalescence(R0, t_end=t_end, storage=storage) for R0 in radii]


def _crossover(r, frac=1.0 / 3.0):
    """First time (in viscous times) at which b reaches frac * R0."""
    for t, b in zip(r["t"], r["b"]):
        if b >= frac * r["R0"]:
            return t / r["tau_visc"]
    return None


def curvature_study(surfaces=(None, 1200.0, 400.0, 200.0, 100.0), *, R0=100.0, t_end=6.0, samples=300,
                    storage="fp32"):
    """Sec. 4, Fig. 8A: coalescence at Oh = 0.286 (R0 = 100, nu = 0.46) on a
    flat surface and on disks of radius Rs. Per surface: the viscous slope,
    the time at which b reaches R0/3 and the final bridge radius."""
    out = []
    for Rs in surfaces:
        r = coalescence(R0, Rs=Rs, t_end=t_end, samples=samples, storage=storage)
        r["t_third"] = _crossover(r)
        r["b_end_over_R0"] = r["b"][-1] / R0
        out.append(r)
    return out


def viscosity_study(nus=(0.16, 0.46, 0.92), surfaces=(None, 100.0), *, R0=100.0, t_end=6.0, samples=300,
                    storage="fp32"):
    """Sec. 4, Fig. 8B: coalescence at several viscosities on a flat surface
    and on a disk of radius 100. Per run: the viscous slope, the time at which
    b reaches R0/3, and the number of times b decreases after its first
    maximum (the oscillations of the inertial regime)."""
    out = []
    for Rs in surfaces:
        for nu in nus:
            r = coalescence(R0, Rs=Rs, t_end=t_end, samples=samples, storage=storage, nu=nu)
            r["t_third"] = _crossover(r)
            b = np.asarray(r["b"])
            r["decreases"] = int(np.sum(np.diff(b) < -1e-3))
            out.append(r)
    return out


def wall_sliding_study(*, nx=400, ny=200, R0=30.0, betas=(0.0, 10.0, 20.0, 30.0, 45.0), thetas=(60.0, 90.0, 120.0),
                       bcs=("martys_chen", "llkc", "virtual_avg"), steps=50000, sample_every=500,
                       storages=("fp32", "fp64")):
    """A droplet of radius R0 tangent to an inclined staircase wall (Sec.
    3.1) for every wall angle, target contact angle (parameters from the
    linear calibration of inputs.wetting_for_angle) and wetting scheme, each
    storage format as one batch. Samples the centre-of-mass sliding velocity
    every ``sample_every`` steps and the contact angle at the end, and reports
    every format's largest deviation from FP64."""
    cases = [(bc, th, be) for bc in bcs for th in thetas for be in betas]
    mask = {be: inputs.inclined_wall_mask(nx, ny, be, R0) for be in betas}
    rA, rB = inputs.sharp_droplet(nx, ny, nx / 2, ny / 2, R0)
    per = {}
    for st in storages:
        sims = []
        for bc, th, be in cases:
            sim = lbm.Simulation(nx, ny, storage=st)
            sim.set_geometry(mask[be]).set_wetting(bc, **inputs.wetting_for_angle(bc, th)).init_fields(rA, rB)
            sims.append(sim)
        batch = lbm.Batch(sims)
        ud = [[] for _ in cases]
        t0 = time.time()
        done = 0
        while done < steps:
            k = min(sample_every, steps - done)
            batch.step(k)
            done += k
            for j, (bc, th, be) in enumerate(cases):
                b = math.radians(be)
                d = sims[j].diagnostics(tangent=(math.cos(b), math.sin(b)))
                ud[j].append(d["sliding_velocity"])
        ang = []
        for j, (bc, th, be) in enumerate(cases):
            wp, wa = wall_line(nx, be, R0, ny)
            ang.append(sims[j].diagnostics(wall_point=wp, wall_angle_deg=wa)["contact_angle_deg"])
        wall = time.time() - t0
        batch.close()
        for sim in sims:
            sim.close()
        per[st] = {"u_d": ud, "theta": ang, "wall_s": wall}
    runs = []
    for j, (bc, th, be) in enumerate(cases):
        r = {"bc": bc, "theta_target": th, "beta": be}
        for st in storages:
            r[f"u_d_end/{st}"] = per[st]["u_d"][j][-1]
            r[f"theta/{st}"] = per[st]["theta"][j]
        if "fp64" in storages:
            for st in storages:
                if st != "fp64":
                    r[f"max_abs_du/{st}"] = float(np.max(np.abs(np.array(per[st]["u_d"][j]) -
                                                                np.array(per["fp64"]["u_d"][j]))))
                    r[f"abs_dtheta/{st}"] = abs(per[st]["theta"][j] - per["fp64"]["theta"][j])
        runs.append(r)
    return {"nx": nx, "ny": ny, "R0": R0, "steps": steps, "sample_every": sample_every,
            "wall_s": {st: per[st]["wall_s"] for st in storages}, "runs": runs,
            "samples": {st: per[st]["u_d"] for st in storages}}


def curved_coalescence_study(*, nx=800, ny=600, Rs=150.0, R0=25.0, gap=52.0, theta=60.0, steps=100000,
                             sample_every=100, storages=("fp64", "fp32", "fp16", "bf16"), delta=8.0):
    """Two droplets of radius R0, centres ``gap`` apart, on a convex disk of
    radius Rs centred in a periodic box (Sec. 4), smoothed interfaces,
    improved scheme at the target contact angle; the bridge radius on the
    symmetry column every ``sample_every`` steps for each storage format and
    its largest deviation from FP64."""
    mask = inputs.circle_surface_mask(nx, ny, nx / 2, ny / 2, Rs, periodic=True)
    yc = ny / 2 + Rs - R0 * math.cos(math.radians(theta))
    rA, rB = inputs.tanh_droplets(nx, ny, (nx / 2 - gap / 2, nx / 2 + gap / 2), yc, R0, 1.0, 0.055, delta)
    rA, rB = rA * (1 - mask), rB * (1 - mask)
    xb = nx // 2
    y0 = next(y for y in range(ny // 2, ny) if mask[y, xb] == 0 and mask[y - 1, xb] == 1)
    wet = inputs.wetting_for_angle("virtual_avg", theta)
    per = {}
    for st in storages:
        sim = lbm.Simulation(nx, ny, periodic_x=True, periodic_y=True, storage=st)
        sim.set_geometry(mask).set_wetting("virtual_avg", **wet).init_fields(rA, rB)
        bs, t0, done = [], time.time(), 0
        while done < steps:
            k = min(sample_every, steps - done)
            sim.step(k)
            done += k
            bs.append(sim.diagnostics(bridge=(xb, y0))["bridge_radius"])
        per[st] = {"b": bs, "wall_s": time.time() - t0, "mass": sim.mass().tolist()}
        sim.close()
    out = {"nx": nx, "ny": ny, "Rs": Rs, "R0": R0, "gap": gap, "theta": theta, "steps": steps,
           "sample_every": sample_every, "bridge": (xb, y0), "b_end": {st: per[st]["b"][-1] for st in storages},
           "wall_s": {st: per[st]["wall_s"] for st in storages}, "mass": {st: per[st]["mass"] for st in storages},
           "b": {st: per[st]["b"] for st in storages}}
    if "fp64" in storages:
        ref = np.array(per["fp64"]["b"])
        out["max_abs_db"] = {st: float(np.max(np.abs(np.array(per[st]["b"]) - ref))) for st in storages
                             if st != "fp64"}
    return out


def _summary_sweep(res):
    rows = []
    for r in res["runs"]:
        last = r["checks"][-1]
        rows.append({"xi": r["xi"], "beta": r["beta"], "theta_deg": round(last["theta_deg"], 2),
                     "theta_prev_deg": round(r["checks"][-2]["theta_deg"], 2) if len(r["checks"]) > 1 else None,
                     "sliding_velocity": last["sliding_velocity"], "max_u": last["max_u"]})
    return {k: v for k, v in res.items() if k != "runs"} | {"table": rows}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp64", "fp16", "bf16"])
    ap.add_argument("--out", default=None, help="write the full result (JSON) here")
    sub = ap.add_subparsers(dest="cmd", required=True)
    a = sub.add_parser("sweep")
    a.add_argument("--n", type=int, default=1000)
    a.add_argument("--R0", type=float, default=100.0)
    a.add_argument("--steps", type=int, default=200000)
    a.add_argument("--check-every", type=int, default=50000)
    a.add_argument("--stencil", type=int, default=25, choices=[9, 25])
    a.add_argument("--xis", type=float, nargs="+", default=[-0.4, -0.2, 0.0, 0.2, 0.4])
    a.add_argument("--betas", type=float, nargs="+", default=[0.0, 10.0, 20.0, 30.0, 45.0])
    c = sub.add_parser("convergence")
    c.add_argument("--radii", type=float, nargs="+", default=[12.5, 25.0, 50.0, 100.0, 200.0, 400.0])
    c.add_argument("--t-end", type=float, default=1.0)
    c.add_argument("--Rs", type=float, default=None)
    cv = sub.add_parser("curvature")
    cv.add_argument("--t-end", type=float, default=6.0)
    vs = sub.add_parser("viscosity")
    vs.add_argument("--t-end", type=float, default=6.0)
    sl = sub.add_parser("slide")
    sl.add_argument("--steps", type=int, default=50000)
    sl.add_argument("--sample-every", type=int, default=500)
    cu = sub.add_parser("curved")
    cu.add_argument("--steps", type=int, default=100000)
    cu.add_argument("--sample-every", type=int, default=100)
    args = ap.parse_args(argv)
    # 128-byte L2 fetches: fastest for the tiled schedule (FP32 single runs) and the batched one
    lbm.set_l2_fetch_granularity(128)
    if args.cmd in ("curvature", "viscosity"):
        res = (curvature_study(t_end=args.t_end, storage=args.storage) if args.cmd == "curvature"
               else viscosity_study(t_end=args.t_end, storage=args.storage))
        summary = [{k: v for k, v in r.items() if k not in ("t", "b", "max_u")} for r in res]
    elif args.cmd == "slide":
        res = wall_sliding_study(steps=args.steps, sample_every=args.sample_every)
        summary = {k: v for k, v in res.items() if k != "samples"}
    elif args.cmd == "curved":
        res = curved_coalescence_study(steps=args.steps, sample_every=args.sample_every)
        summary = {k: v for k, v in res.items() if k != "b"}
    elif args.cmd == "sweep":
        res = contact_angle_sweep(args.xis, args.betas, n=args.n, R0=args.R0, steps=args.steps,
                                  check_every=args.check_every, avg_stencil=args.stencil, storage=args.storage)
        summary = _summary_sweep(res)
    else:
        res = [coalescence(R0, Rs=args.Rs, t_end=args.t_end, storage=args.storage) for R0 in args.radii]
        summary = [{k: v for k, v in r.items() if k not in ("t", "b", "max_u")} for r in res]
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(res, fh)
    json.dump(summary, sys.stdout, indent=1)
    print()


if __name__ == "__main__":
    main()
