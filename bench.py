"""Benchmark of the implicit-FDTD PIC particle cycle on GB300 (one JSON line on stdout).

Workload (default): 2048 x 512 periodic grid, CFL 1, theta 1/2, order-2 shapes, drifting
pair plasma gamma0 = 40 with 1e-3 rest-frame spread, 32 macro-particles per cell per
species (67,108,864 particles), seeded synthetic inputs. A step is one pass of the whole
particle cycle: gather, Boris push, move, Esirkepov deposit, Eq. (7) PCG solve to 1e-10,
E/B update. The chosen form is MIXED32 (int cell + FP32 offset particles, FP32
gather/push/deposit in shared-memory tiles, FP64 field solve); the plain FP64 GPU path is
timed beside it on the same inputs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched under torchrun) every rank runs an independent replica with its own
seed (the path has no data-path exchange on one grid); value = particles of all ranks x K
/ the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle updates/s and field-solve ms/step on 1 GB300, chosen vs plain FP64"
UNIT = "particle updates/s"
WORKLOADS = {
    # name: (nx, ny, ppc per species, order, gamma0, u_th, cfl, theta, seed)
    "cfg2": (2048, 512, 32, 2, 40.0, 1e-3, 1.0, 0.5, 2),
    "cfg1": (64, 64, 8, 1, 20.0, 1e-3, 1.0, 0.5, 1),
    # a quarter of cfg2 (same density and physics, 16.8M particles): profiling captures
    "cfg2q": (1024, 256, 32, 2, 40.0, 1e-3, 1.0, 0.5, 2),
}
FP32_BYTES_PER_PARTICLE = 48  # 24 B read + 24 B written per MIXED32 particle update
FP32_BYTES_PER_CELL = 36      # 6 FP32 field components read, 3 FP32 currents written
FP64_BYTES_PER_PARTICLE = 80  # 40 B read + 40 B written per FP64 particle update
FP64_BYTES_PER_CELL = 72


def describe(name):
    nx, ny, ppc, order, g0, uth, cfl, theta, seed = WORKLOADS[name]
    return (f"{nx}x{ny} periodic, CFL {cfl}, theta {theta}, order {order}, pair plasma "
            f"gamma0 {g0:g}, u_th {uth:g}, {ppc} ppc/species ({2 * nx * ny * ppc} particles), "
            f"PCG rtol 1e-10")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            v = [x.strip() for x in line.split(",")]
            if len(v) < 9:
                continue
            try:
                sm.append(float(v[1]))
                mx.append(float(v[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if v[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_for(kernel_key):
    """Per-launch DRAM bytes of a kernel from the committed ncu summary, only while the
    kernel source is unchanged since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(kernel_key)
    if not d:
        return None
    h = hashlib.sha256(open(os.path.join(ROOT, d["source"]), "rb").read()).hexdigest()[:16]
    return d["bytes_per_launch"] if h == d["source_sha"] else None


def make_inputs(name, seed_offset=0, pinned=False):
    from paper_1412_2480_gb300 import inputs
    nx, ny, ppc, order, g0, uth, cfl, theta, seed = WORKLOADS[name]
    w, sp = inputs.drifting_pair_plasma(nx, ny, ppc, g0, uth, seed + seed_offset)
    if pinned:
        import torch
        out = []
        for d in sp:
            e = {"qm": d["qm"]}
            for k in ("x", "y", "ux", "uy", "uz"):
                t = torch.empty(d[k].size, dtype=torch.float64, pin_memory=True)
                t.numpy()[:] = d[k]
                e[k] = t.numpy()
            out.append(e)
        sp = out
    return w, sp


NO_GRAPH = False  # --no-graph: direct launches (profilers skip kernels of conditional graphs)


def new_sim(name, precision, stream=None):
    import paper_1412_2480_gb300 as pic
    nx, ny, ppc, order, g0, uth, cfl, theta, seed = WORKLOADS[name]
    prm = pic.pic_params_default(nx=nx, ny=ny, cfl=cfl, theta=theta, shape_order=order, gamma0=g0,
                                 ppc=ppc, precision=precision, cg_rtol=1e-10, cg_max_iter=200,
                                 flags=pic.PIC_NO_GRAPH if NO_GRAPH else 0)
    h = pic.pic_init(prm)
    if stream is not None:
        pic.pic_set_stream(h, stream)
    return h


def load(h, sp):
    import paper_1412_2480_gb300 as pic
    for s, d in enumerate(sp):
        pic.pic_load_particles(h, s, d["x"], d["y"], d["ux"], d["uy"], d["uz"])


def launches_per_step(precision):
    # kernels of ours per step besides the PCG loop (2 kernels per PCG iteration):
    # step_begin, [FP64: push x2 | MIXED32: push_overflow, clear_overflow, push_tile,
    # migrate], zero_x, rhs, update_E, update_B, step_end
    return 7 if precision == 0 else 9


def run_ours(args, dist):
    import torch

    import paper_1412_2480_gb300 as pic
    rank, world = dist["rank"], dist["world"]
    dev = dist["local_rank"]
    torch.cuda.set_device(dev)
    name = args.workload
    nx, ny, ppc, order, g0, uth, cfl, theta, seed = WORKLOADS[name]
    npart = 2 * nx * ny * ppc
    stream = torch.cuda.Stream()
    w, sp = make_inputs(name, seed_offset=rank, pinned=True)
    prec = pic.PIC_MIXED32 if args.precision == "mixed" else pic.PIC_FP64

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def max_over_ranks(v):
        if world == 1:
            return v
        t = torch.tensor([v], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    # ---- end to end through the C ABI with host buffers: load (H2D) + K steps +
    # per-step moments (D2H) + final field readback (D2H) ----
    h = new_sim(name, prec, stream)
    out_fields = torch.empty(nx * ny, dtype=torch.float64, pin_memory=True).numpy()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    load(h, sp)
    for _ in range(args.steps):
        pic.pic_step(h, 1)
        pic.pic_moments(h)
    for c in range(6):
        pic.pic_fields(h, c, out_fields)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    barrier()
    h2d = npart * 5 * 8 / args.steps
    d2h = (6 * nx * ny * 8) / args.steps + 160
    pic.pic_free(h)

    # ---- device-timed steps with inputs resident ----
    h = new_sim(name, prec, stream)
    load(h, sp)
    pic.pic_step(h, args.warmup)
    m0 = pic.pic_moments(h)
    clocks = Clocks(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0.record(stream)
    pic.pic_step(h, args.steps)
    ev1.record(stream)
    ev1.synchronize()
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ms)
    barrier()
    m1 = pic.pic_moments(h)
    cg_iters = (m1["cg_iters_total"] - m0["cg_iters_total"]) / args.steps
    launches = int(args.steps * launches_per_step(prec) + 2 * (m1["cg_iters_total"] - m0["cg_iters_total"]))
    # ---- per-phase CUDA-event timing (profiling graph) ----
    prof = pic.pic_profile(h, args.prof_steps)
    pic.pic_free(h)

    res = {"ms": ms_max, "prof": prof, "cg_iters": cg_iters, "clocks": ck, "launches": launches,
           "e2e_s": e2e_s, "h2d": h2d, "d2h": d2h, "npart": npart, "rtol_reached": m1["cg_rel_resid"]}

    # ---- plain FP64 GPU path on the same inputs (comparison leg) ----
    if prec == pic.PIC_MIXED32 and not args.skip_fp64 and rank == 0:
        h = new_sim(name, pic.PIC_FP64, stream)
        load(h, sp)
        pic.pic_step(h, 2)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        k64 = max(2, args.steps // 4)
        e0.record(stream)
        pic.pic_step(h, k64)
        e1.record(stream)
        e1.synchronize()
        ms64 = e0.elapsed_time(e1) / k64
        prof64 = pic.pic_profile(h, 2)
        pic.pic_free(h)
        res["fp64"] = {"ms_per_step": ms64, "value": npart / (ms64 * 1e-3),
                       "field_solve_ms_per_step": prof64["field_ms"],
                       "push_kernel_ms": prof64["push_kernel_ms"], "steps": k64}
    return res


def oracle_sample(name, seconds_target=12.0):
    """The CPU oracle as it stands, on a bounded sample of the workload: the same
    physics on a (nx/8) x (ny/8) periodic patch with the same particles per cell,
    timed over whole steps on one host core."""
    import oracle
    from paper_1412_2480_gb300 import inputs
    nx, ny, ppc, order, g0, uth, cfl, theta, seed = WORKLOADS[name]
    sx, sy = max(16, nx // 8), max(16, ny // 8)
    w, sp = inputs.drifting_pair_plasma(sx, sy, ppc, g0, uth, seed)
    species = [oracle.Species(d["qm"], w, d["x"], d["y"], d["ux"], d["uy"], d["uz"]) for d in sp]
    sim = oracle.OracleSim(sx, sy, cfl, theta, order, species, cg_rtol=1e-10)
    oracle.build()
    steps, t = 0, 0.0
    while t < seconds_target and steps < 50:
        t0 = time.perf_counter()
        sim.step(1)
        t += time.perf_counter() - t0
        steps += 1
    npart = 2 * sx * sy * ppc
    return {"value": npart * steps / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{sx}x{sy} patch of the workload ({npart} particles, same ppc/order/gamma0), "
                      f"{steps} whole steps in {t:.1f} s on 1 host core"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="cfg2")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--prof-steps", type=int, default=4)
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch kernels directly (for profiler launch lists), not a bench number")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    global NO_GRAPH
    NO_GRAPH = args.no_graph

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    dist = {"world": world, "rank": rank, "local_rank": local_rank}

    if args.impl == "reference":
        if rank != 0:
            return
        # the oracle is the reference arm: a bounded sample per step, on host cores
        per = []
        for _ in range(args.warmup):
            oracle_sample(args.workload, seconds_target=2.0)
        for _ in range(args.steps):
            per.append(oracle_sample(args.workload, seconds_target=3.0))
        v = statistics.median(p["value"] for p in per)
        cpu = dict(per[-1])
        cpu["value"] = v
        nx, ny, ppc = WORKLOADS[args.workload][:3]
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 2 * nx * ny * ppc / v * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": describe(args.workload), "l2": "n/a (host)"},
                "cpu_baseline": cpu,
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(args.workload)
    res = run_ours(args, dist)
    if rank != 0:
        return
    import paper_1412_2480_gb300 as pic  # noqa: F401
    nx, ny, ppc = WORKLOADS[args.workload][:3]
    npart = res["npart"]
    value = world * npart * args.steps / (res["ms"] * 1e-3)
    hbm, src = peaks()
    mixed = args.precision == "mixed"
    bpp = FP32_BYTES_PER_PARTICLE if mixed else FP64_BYTES_PER_PARTICLE
    bpc = FP32_BYTES_PER_CELL if mixed else FP64_BYTES_PER_CELL
    alg_bytes = bpp * npart + bpc * nx * ny
    kms = res["prof"]["push_kernel_ms"]
    achieved = alg_bytes / (kms * 1e-3) / 1e9
    key = "k_push_tile" if mixed else "k_push_fp64"
    traffic = traffic_for(f"{key}:{args.workload}")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if mixed else "f64",
        "data": "synthetic",
        "config": {"workload": describe(args.workload),
                   "form": "MIXED32 (int cell + FP32 offset; FP32 gather/push/deposit; FP64 PCG and field update)"
                   if mixed else "FP64",
                   "l2": "inputs larger than L2 (particle state 1.6 GB MIXED32 / 2.7 GB FP64)",
                   "replicas": world},
        "field_solve_ms_per_step": res["prof"]["field_ms"],
        "particle_ms_per_step": res["prof"]["particle_ms"],
        "cg_iters_per_step": res["cg_iters"],
        "e2e": {"value": world * npart * args.steps / res["e2e_s"], "unit": UNIT,
                "h2d_bytes_per_step": int(res["h2d"]), "d2h_bytes_per_step": int(res["d2h"]),
                "what": "pic_load_particles from pinned host arrays + K x (pic_step(1) + pic_moments) + pic_fields x 6"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic, "kernel": key,
                     "peak_source": src,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "kernel_ms": kms},
        "gpu_launches": res["launches"],
        "clocks": res["clocks"],
    }
    if "fp64" in res:
        line["plain_fp64"] = res["fp64"]
        line["speedup_vs_plain_fp64"] = res["fp64"]["ms_per_step"] / (res["ms"] / args.steps)
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
