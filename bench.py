#!/usr/bin/env python
"""Throughput benchmark of the two-component Shan-Chen D2Q9 step with the
improved virtual-density wetting condition on one GB300.

Workload: 8192 x 8192 fully periodic porous medium of non-overlapping disks
(radius uniform in [8, 40], solid fraction 0.40, seed 1) with sharp droplets
of the majority component (radius uniform in [8, 32]) filling 30% of the
pore space (seed 2); G_AB = 3, tau = 1, improved virtual-density scheme with
xi = -0.2. One bench step is one time step over the whole grid. The metric
is MLUPS counted over fluid nodes.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line. With --gpus N (under torchrun) every rank runs an
independent replica on its own GPU (the method has no exchange between
independent simulations): value = all ranks' fluid-node updates / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % HBM roofline at 1 GB300 (FP32 vs FP16-storage vs batched), err vs FP64"
BYTES_PER_UPDATE = {"fp32": 144, "fp64": 288, "fp16": 72, "bf16": 72}
XI = -0.2  # the paper's coalescence runs (theta = 71 deg)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


from paper_2009_12584_gb300.experiments import chi_from_xi  # noqa: E402  (xi -> chi reading)


def workload(n, cache=True):
    from paper_2009_12584_gb300 import inputs
    path = os.path.join(tempfile.gettempdir(), f"lbm_porous_{n}_v1.npz")
    if cache and os.path.exists(path):
        d = np.load(path)
        return d["mask"], d["rA"], d["rB"]
    t0 = time.time()
    mask = inputs.porous_disks(n, n, solid_fraction=0.40, rmin=8, rmax=40, seed=1)
    rA, rB = inputs.pore_droplets(mask, a_fraction=0.30, rmin=8, rmax=32, seed=2)
    log(f"[bench] generated {n}^2 porous workload in {time.time() - t0:.1f}s")
    if cache:
        try:
            np.savez(path, mask=mask, rA=rA, rB=rB)
        except OSError:
            pass
    return mask, rA, rB


def source_hash():
    """Hash of the CUDA sources' code: comments and whitespace are dropped,
    so that a change of wording does not invalidate the recorded traffic,
    and every change of code does."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2009_12584_gb300", "csrc")
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh")):
            text = open(os.path.join(d, name), encoding="utf-8").read()
            text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
            text = re.sub(r"//[^\n]*", " ", text)
            h.update(name.encode() + b"\0" + " ".join(text.split()).encode())
    return h.hexdigest()[:16]


def effective_schedule(kernel, storage):
    """The schedule lbm_step runs on the benchmark workload (improved scheme):
    AUTO takes the tiled one for 4- and 8-byte storage (the halo one only
    under the one-node-reach schemes) and the two-pass one for 16-bit
    storage; 16-bit storage runs a FUSED choice as two-pass too (the
    marching kernel has no 16-bit path)."""
    if storage in ("fp16", "bf16"):
        return "tiled" if kernel == "tiled" else "two_pass"
    return "tiled" if kernel == "auto" else kernel


def l2_fetch_for(kernel, storage, requested):
    """The L2 fetch granularity an arm runs with: the one requested, else the
    one each schedule runs best with (the tiled kernel's scattered ring reads
    gain from 128-byte fetches, the two-pass pulls from 32-byte ones)."""
    if requested >= 0:
        return requested
    return 128 if effective_schedule(kernel, storage) == "tiled" else 32


def measured_traffic(kernel_class, storage, l2_fetch):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources with the same L2 fetch granularity (else
    None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None
    e = d.get(f"{kernel_class}/{storage}")
    if not e or e.get("source_hash") != source_hash() or e.get("l2_fetch_granularity_bytes") != l2_fetch:
        return None
    return e.get("bytes_per_launch_full")


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.flush()
        rows = []
        for line in open(self.out.name):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), max=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], pcap=parts[8]))
            except ValueError:
                continue
        os.unlink(self.out.name)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for k, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                            ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[k].lower() == "active":
                    reasons.add(name)
        sm = sorted(r["sm"] for r in rows)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r["max"] for r in rows),
                "power_w_max": max(r["power"] for r in rows), "samples": len(rows),
                "reasons": sorted(reasons)}


def host_description():
    """nproc and the CPU model of this host (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        fields = {}
        for line in out.splitlines():
            if ":" in line:
                k, v = line.split(":", 1)
                fields.setdefault(k.strip(), v.strip())
        model = fields.get("Model name") or fields.get("Vendor ID")
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    import platform
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or "unknown",
            "machine": platform.machine()}


def _oracle_rate(mask, rA, rB, threads, target_s, periodic=True, **kw):
    """Fluid-node MLUPS of the oracle, as it stands, with `threads` OpenMP
    threads (0: one per core) on one bounded sample; (rate, steps, seconds,
    threads used)."""
    import oracle
    used = oracle.set_threads(threads)
    ny, nx = mask.shape
    o = oracle.Oracle(nx, ny, mask, periodic_x=periodic, periodic_y=periodic, **kw).init(rA, rB)
    t0 = time.perf_counter()
    o.step(1)
    per = time.perf_counter() - t0
    steps = max(2, int(target_s / max(per, 1e-4)))
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    nf = int((mask == 0).sum())
    return nf * steps / dt / 1e6, steps, dt, used


def cpu_baseline(target_s=8.0):
    """The FP64 oracle, as it stands, timed on this host's cores: a 512 x 512
    periodic porous medium drawn with the benchmark's recipe (seeds 1/2),
    improved scheme, single thread and with one OpenMP thread per core (the
    node loops in parallel; results bit for bit those of one thread), and the
    400 x 200 inclined-plane set-up of Sec. 3.1 (R0 = 30, beta = 20 deg,
    improved scheme) on all cores."""
    import oracle
    from paper_2009_12584_gb300 import inputs
    n = 512
    mask = inputs.porous_disks(n, n, solid_fraction=0.40, rmin=8, rmax=40, seed=1)
    rA, rB = inputs.pore_droplets(mask, a_fraction=0.30, rmin=8, rmax=32, seed=2)
    kw = dict(bc=oracle.BC_VIRTUAL_AVG, G_s=(3.0, 3.0), chi=chi_from_xi(XI))
    r1, s1, d1, _ = _oracle_rate(mask, rA, rB, 1, target_s, **kw)
    ra, sa, da, threads = _oracle_rate(mask, rA, rB, 0, target_s, **kw)
    m2 = inputs.inclined_wall_mask(400, 200, 20.0, 30)
    a2, b2 = inputs.sharp_droplet(400, 200, 200, 100, 30)
    rc, sc, dc, _ = _oracle_rate(m2, a2, b2, 0, target_s, periodic=False, **kw)
    oracle.set_threads(0)
    return {"value": round(ra, 3), "unit": "MLUPS", "cores": threads, "kind": "oracle",
            "sample": f"{n}x{n} periodic porous medium (same recipe, seeds 1/2), improved BC, FP64, "
                      f"{sa} steps in {da:.1f} s on {threads} OpenMP threads",
            "single_thread": {"value": round(r1, 3), "unit": "MLUPS", "cores": 1,
                              "sample": f"same medium, {s1} steps in {d1:.1f} s"},
            "inclined_plane_400x200": {"value": round(rc, 3), "unit": "MLUPS", "cores": threads,
                                       "sample": f"Sec. 3.1 set-up, R0 = 30, beta = 20 deg, improved BC, "
                                                 f"{sc} steps in {dc:.1f} s"},
            "host": host_description()}


def max_over_ranks(x: float, world: int, device="cuda") -> float:
    """The largest value of x over all ranks (the job ends with its slowest
    rank); x itself on one rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_mlups(fluid_nodes: int, steps: int, seconds: float, world: int) -> float:
    """Whole-job MLUPS of `world` replicas that each advance `fluid_nodes`
    nodes `steps` times, timed by the slowest rank."""
    return world * fluid_nodes * steps / seconds / 1e6


def run_reference(args, rank):
    """Reference arm: the FP64 oracle timed on the host cores."""
    if rank != 0:
        return
    import oracle
    from paper_2009_12584_gb300 import inputs
    cores = oracle.set_threads(0)  # one OpenMP thread per core
    probe = 128
    m = inputs.porous_disks(probe, probe, 0.40, 8, 40, seed=1)
    a, b = inputs.pore_droplets(m, 0.30, 8, 32, seed=2)
    o = oracle.Oracle(probe, probe, m, periodic_x=True, periodic_y=True, bc=oracle.BC_VIRTUAL_AVG,
                      G_s=(3.0, 3.0), chi=chi_from_xi(XI)).init(a, b)
    t0 = time.perf_counter()
    o.step(2)
    rate = probe * probe * 2 / (time.perf_counter() - t0)
    budget = 120.0
    side = int(np.sqrt(budget * rate / max(1, args.steps + args.warmup)))
    side = int(max(64, min(1024, side)))
    mask = inputs.porous_disks(side, side, 0.40, 8, 40, seed=1)
    rA, rB = inputs.pore_droplets(mask, 0.30, 8, 32, seed=2)
    o = oracle.Oracle(side, side, mask, periodic_x=True, periodic_y=True, bc=oracle.BC_VIRTUAL_AVG,
                      G_s=(3.0, 3.0), chi=chi_from_xi(XI)).init(rA, rB)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    nf = int((mask == 0).sum())
    v = nf * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"porous medium {side}x{side} sample of the 8192x8192 recipe",
                       "nx": side, "ny": side, "fluid_nodes": nf, "bc": "virtual_avg", "storage": "fp64"},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": f"{side}x{side} porous medium, same recipe, {args.steps} steps, "
                                       f"{cores} OpenMP threads", "host": host_description()},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_single(n, mask, rA, rB, nf, storage, kernel, steps, warmup, l2_fetch, velocity_refs=False):
    """The throughput workload with another population storage (16-bit
    storage: velocity_refs selects the encoding relative to the writer's
    momentum, lbm_params.velocity_refs)."""
    import torch
    from paper_2009_12584_gb300 import lbm
    l2_prev = lbm.set_l2_fetch_granularity(l2_fetch) if l2_fetch else None
    sim = lbm.Simulation(n, n, periodic_x=True, periodic_y=True, storage=storage, kernel=kernel,
                         velocity_refs=velocity_refs)
    sim.set_geometry(mask).set_wetting("virtual_avg", G_s=(3.0, 3.0), chi=chi_from_xi(XI)).init_fields(rA, rB)
    sim.step(warmup)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ms_cls, cnt_cls = sim.step_profiled(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t_ms = e0.elapsed_time(e1)
    dom = max(ms_cls, key=lambda k: ms_cls[k])
    per_launch = ms_cls[dom] / max(1, cnt_cls[dom])
    bpu = BYTES_PER_UPDATE[storage] if dom in ("fused", "collide") else BYTES_PER_UPDATE[storage] // 2
    pk, _ = peaks()
    ach = bpu * nf / (per_launch / 1e3) / 1e9
    out = {"value": round(nf * steps / (t_ms / 1e3) / 1e6, 1), "unit": "MLUPS", "ms_per_step": round(t_ms / steps, 4),
           "roofline": {"kernel": dom, "achieved": round(ach, 1), "frac": round(ach / pk["hbm_gbs"], 4),
                        "algorithmic_bytes_per_update": bpu},
           "kernel_ms_per_step": {k: round(v / steps, 4) for k, v in ms_cls.items() if cnt_cls[k]},
           "l2_fetch_granularity_bytes": l2_fetch}
    del sim
    torch.cuda.empty_cache()
    if l2_prev is not None:
        lbm.set_l2_fetch_granularity(l2_prev)
    return out


def run_batched(storage, steps, warmup, nsims=512, l2_fetch=128):
    """512 independent inclined-wall simulations (sizes 64x64 ... 512x256,
    wall angle 0 ... 45 deg, contact angle 45 ... 135 deg, three schemes mixed,
    seed 0) advanced together by one batch; steps per graph replay and
    threads per block picked by the autotuner. Their single straight walls
    leave long fluid segments, which stream best with 128-byte L2 fetches
    (the porous arms use 32); the previous setting is restored after."""
    import torch
    from paper_2009_12584_gb300 import inputs, lbm
    l2_prev = lbm.set_l2_fetch_granularity(l2_fetch)
    t0 = time.time()
    work = inputs.batched_workload(nsims, seed=0)
    sims = []
    nf = 0
    for w in work:
        s = lbm.Simulation(w["nx"], w["ny"], storage=storage)
        s.set_geometry(w["mask"]).set_wetting(w["bc"], **w["wetting"]).init_fields(w["rhoA"], w["rhoB"])
        nf += int((w["mask"] == 0).sum())
        sims.append(s)
    b = lbm.Batch(sims)
    choice = b.autotune(16)
    b.step(max(warmup, 2))
    torch.cuda.synchronize()
    setup = time.time() - t0
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = b.launch_count
    e0.record(stream)
    b.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t_ms = e0.elapsed_time(e1)
    launches = b.launch_count - l0
    sched = b.config()[0]
    # the schedule the autotuner did not keep, timed the same way after the
    # measured steps (for the record; it does not enter the value)
    others = {}
    for other in ("two_pass", "tiled"):
        if other == sched or (other == "tiled" and storage not in ("fp32", "fp64")):
            continue
        b.set_schedule(other)
        b.step(2)
        e0.record(stream)
        b.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        others[other] = round(nf * steps / (e0.elapsed_time(e1) / 1e3) / 1e6, 1)
    out = {"value": round(nf * steps / (t_ms / 1e3) / 1e6, 1), "unit": "MLUPS", "ms_per_step": round(t_ms / steps, 4),
           "sims": nsims, "fluid_nodes": nf, "schedule": sched, "threads_per_block": choice[0],
           "steps_per_graph": choice[1], "other_schedules_mlups": others,
           "gpu_launches": launches, "setup_s": round(setup, 1),
           "workload": "512 inclined-wall simulations, 64x64..512x256, beta U[0,45], theta U[45,135], "
                       "MC/LLKC/improved mixed, seed 0", "l2_fetch_granularity_bytes": l2_fetch}
    b.close()
    del sims, b
    torch.cuda.empty_cache()
    lbm.set_l2_fetch_granularity(l2_prev)
    return out


def accuracy():
    """Error of each storage format against the FP64 oracle: the values in
    tests/golden/oracle_accuracy.json, written from the oracle alone by
    tests/golden/make_oracle_accuracy.py, on the inclined-plane set-up of
    Sec. 3.1 at 400 x 200 (R0 = 30; Martys-Chen G_w = -0.2, LLKC G_w = -0.5,
    improved xi = -0.2; beta = 0 and 20 deg; 10,000 steps): the sliding
    velocity every 1,000 steps and the final contact angle, measured on the
    device (lbm_diagnostics). Bounds: 1e-6 and 0.5 deg."""
    import math
    import torch
    from paper_2009_12584_gb300 import inputs, lbm
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "oracle_accuracy.json")))
    wet = {"mc": ("martys_chen", dict(G_s=(-0.2, 0.2))), "llkc": ("llkc", dict(G_s=(-0.5, 0.5))),
           "improved": ("virtual_avg", dict(G_s=(3.0, 3.0), chi=(1.2, 0.8)))}
    nx, ny, R0 = gold["nx"], gold["ny"], gold["R0"]
    res = {"reference": "FP64 oracle (tests/golden/oracle_accuracy.json)", "bounds": {"sliding_velocity": 1e-6,
                                                                                     "contact_angle_deg": 0.5}}
    worst = {}
    for c in gold["cases"]:
        b = math.radians(c["beta"])
        mask = inputs.inclined_wall_mask(nx, ny, c["beta"], R0)
        rA, rB = inputs.sharp_droplet(nx, ny, nx / 2, ny / 2, R0)
        dkw = dict(level=gold["level"], rho_out=gold["rho_out"], tangent=(math.cos(b), math.sin(b)),
                   wall_point=(nx / 2 + R0 * math.sin(b), ny / 2 - R0 * math.cos(b)), wall_angle_deg=c["beta"],
                   exclude=gold["exclude"], box=tuple(gold["box"]))
        angle = c["beta"] == 0.0 or c["scheme"] == "improved"  # sliding droplets reach the box
        for st in ("fp32", "fp16", "fp16u", "bf16", "bf16u"):
            kind, wkw = wet[c["scheme"]]
            # "u": 16-bit storage with velocity references (lbm_params.velocity_refs)
            sim = lbm.Simulation(nx, ny, storage=st.rstrip("u"), velocity_refs=st.endswith("u"))
            sim.set_geometry(mask).set_wetting(kind, **wkw).init_fields(rA, rB)
            dud = 0.0
            for ud in c["sliding_velocity"]:
                sim.step(c["every"])
                d = sim.diagnostics(**dkw)
                dud = max(dud, abs(d["sliding_velocity"] - ud))
            dth = abs(d["contact_angle_deg"] - c["contact_angle_deg"]) if angle else None
            res[f"{c['scheme']}/beta{int(c['beta'])}/{st}"] = {
                "max_abs_err_sliding_velocity": dud, "sliding_velocity_end": d["sliding_velocity"],
                "sliding_velocity_end_oracle": c["sliding_velocity"][-1],
                "contact_angle_deg": d["contact_angle_deg"] if angle else None,
                "contact_angle_deg_oracle": c["contact_angle_deg"] if angle else None, "abs_err_deg": dth}
            w = worst.setdefault(st, {"max_abs_err_sliding_velocity": 0.0, "max_abs_err_deg": 0.0})
            w["max_abs_err_sliding_velocity"] = max(w["max_abs_err_sliding_velocity"], dud)
            if dth is not None:
                w["max_abs_err_deg"] = max(w["max_abs_err_deg"], dth)
            sim.close()
    for st, w in worst.items():
        w["meets_bounds"] = w["max_abs_err_sliding_velocity"] <= 1e-6 and w["max_abs_err_deg"] <= 0.5
    res["worst"] = worst
    torch.cuda.empty_cache()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp64", "fp16", "bf16"])
    ap.add_argument("--kernel", default="auto", choices=["auto", "two_pass", "fused", "tiled", "halo", "tma"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the fp16/bf16, batched and accuracy arms")
    ap.add_argument("--l2-fetch", type=int, default=-1, choices=[-1, 0, 32, 64, 128],
                    help="L2 fetch granularity hint for this process (0: leave the CUDA default; "
                         "-1: per schedule, 128 bytes for the tiled one and 32 for the two-pass one)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist
    from paper_2009_12584_gb300 import build, lbm

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    l2_fetch = l2_fetch_for(args.kernel, args.storage, args.l2_fetch)
    l2_prev = lbm.set_l2_fetch_granularity(l2_fetch) if l2_fetch else None

    n = args.n
    mask, rA, rB = workload(n)
    nf = int((mask == 0).sum())
    chi = chi_from_xi(XI)
    sim = lbm.Simulation(n, n, periodic_x=True, periodic_y=True, storage=args.storage, kernel=args.kernel)
    sim.set_geometry(mask).set_wetting("virtual_avg", G_s=(3.0, 3.0), chi=chi).init_fields(rA, rB)
    stream = torch.cuda.current_stream()
    sim.step(args.warmup)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v for v in vis.split(",") if v.strip()]
    sampler = ClockSampler(ids[local] if local < len(ids) else local)
    sampler.start()
    time.sleep(0.4)
    l0 = sim.launch_count
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ms_cls, cnt_cls = sim.step_profiled(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = sim.launch_count - l0
    clocks = sampler.stop()
    t_ms = max_over_ranks(e0.elapsed_time(e1), world)
    if world > 1:
        dist.barrier()
    ms_per_step = t_ms / args.steps
    value = replica_mlups(nf, args.steps, t_ms / 1e3, world)

    # dominant kernel and its roofline
    dom = max(ms_cls, key=lambda k: ms_cls[k])
    per_launch_ms = ms_cls[dom] / max(1, cnt_cls[dom])
    bpu = BYTES_PER_UPDATE[args.storage] if dom in ("fused", "collide") else BYTES_PER_UPDATE[args.storage] // 2
    alg_bytes = bpu * nf
    achieved = alg_bytes / (per_launch_ms / 1e3) / 1e9
    pk, pk_kind = peaks()
    # the single-pass class is k_tile under AUTO and TILED (4- and 8-byte
    # storage), k_march under FUSED, k_halo under HALO, k_tile_tma under TMA
    sched = effective_schedule(args.kernel, args.storage)
    tkey = dom if dom != "fused" else {"tiled": "tile", "fused": "march"}.get(sched, sched)
    traffic = measured_traffic(tkey, args.storage, l2_fetch)
    kernel_name = {"tile": "k_tile", "march": "k_march", "halo": "k_halo", "tma": "k_tile_tma",
                   "collide": "k_collide_list", "density": "k_density_list"}.get(tkey, tkey)
    roofline = {"bound": "hbm", "kernel": dom, "kernel_name": kernel_name, "achieved": round(achieved, 1),
                "peak": pk["hbm_gbs"],
                "peak_kind": pk_kind, "unit": "GB/s", "frac": round(achieved / pk["hbm_gbs"], 4),
                "traffic": traffic, "algorithmic_bytes_per_launch": alg_bytes,
                "algorithmic_bytes_per_update": bpu,
                "traffic_bytes_per_update": None if traffic is None else round(traffic / nf, 1),
                "per_launch_ms": round(per_launch_ms, 4),
                "kernel_ms_per_step": {k: round(v / args.steps, 4) for k, v in ms_cls.items() if cnt_cls[k]}}

    # end to end through the host API: host buffers in, host buffers out
    # (every rank runs it; the slowest rank's wall time counts)
    e2e = None
    if not args.no_e2e:
        # the FP32 host interface (lbm_run_host_f32): the initial densities are
        # FP32 arrays here, the moments come back as FP32
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        h_mask, h_rA, h_rB = pin(mask), pin(rA.astype(np.float32)), pin(rB.astype(np.float32))
        outs = [torch.empty((n, n), dtype=torch.float32).pin_memory() for _ in range(4)]
        sim2 = sim  # reuse the context and its workspace
        # one untimed call first (like the warm-up steps of the device-timed arm)
        sim2.run_host_f32(sim.wetting, h_mask, h_rA, h_rB, args.warmup, outs)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        sim2.run_host_f32(sim.wetting, h_mask, h_rA, h_rB, args.steps, outs)
        t_e2e = max_over_ranks(time.perf_counter() - t0, world)
        h2d = world * (h_mask.numel() + h_rA.numel() * 4 + h_rB.numel() * 4)  # whole job, like the value
        d2h = world * sum(o.numel() * 4 for o in outs)
        e2e = {"value": replica_mlups(nf, args.steps, t_e2e, world), "unit": "MLUPS",
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "wall_s": round(t_e2e, 3),
               "what": "lbm_run_host_f32: mask + FP32 densities H2D, geometry, init, K steps, FP32 moments D2H"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()

    # the other arms of the metric: 16-bit storage and batched simulations
    extra = {}
    if rank == 0 and not args.no_extra:
        del sim
        torch.cuda.empty_cache()
        # 16-bit storage, both encodings ("u": relative to the writer's
        # momentum, the encoding that holds the accuracy bounds)
        for st in ("fp16", "bf16", "fp16u", "bf16u"):
            base = st.rstrip("u")
            extra[st] = run_single(n, mask, rA, rB, nf, base, args.kernel, args.steps, args.warmup,
                                   l2_fetch_for(args.kernel, base, args.l2_fetch), velocity_refs=st.endswith("u"))
        for st in ("fp32", "fp16"):
            extra[f"batched_{st}"] = run_batched(st, args.steps, args.warmup)
        extra["err_vs_oracle"] = accuracy()

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp32": "f32", "fp64": "f64", "fp16": "f32 (fp16 storage)",
                          "bf16": "f32 (bf16 storage)"}[args.storage],
                "data": "synthetic",
                "config": {"workload": f"porous medium {n}x{n}, improved virtual-density BC, {args.storage}",
                           "nx": n, "ny": n, "fluid_nodes": nf, "solid_fraction": round(1 - nf / n / n, 4),
                           "bc": "virtual_avg", "xi": XI, "chi": chi, "tau": 1.0, "G_AB": 3.0,
                           "storage": args.storage, "kernel": args.kernel,
                           "schedule": effective_schedule(args.kernel, args.storage),
                           "l2": "inputs larger than L2 (populations %.1f GB per buffer)"
                                 % (18 * n * n * BYTES_PER_UPDATE[args.storage] / 144 * 4 / 1e9),
                           "all_node_mlups": round(world * n * n * args.steps / (t_ms / 1e3) / 1e6, 1),
                           "parallelism": f"replicas x{world}",
                           "l2_fetch_granularity_bytes": l2_fetch or l2_prev},
                "roofline": roofline, "gpu_launches": launches, "clocks": clocks, "e2e": e2e,
                "cpu_baseline": cpu, **extra}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
