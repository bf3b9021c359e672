"""Benchmark of the implicit-FDTD PIC particle cycle on GB300 (one JSON line on stdout).

Workload (default, cfg2): 2048 x 512 periodic grid, CFL 1, theta 1/2, order-2 shapes,
drifting pair plasma gamma0 = 40 with 1e-3 rest-frame spread, 32 macro-particles per cell
per species (67,108,864 particles), seeded synthetic inputs. A step is one pass of the
whole particle cycle: gather, Boris push, move, Esirkepov deposit, Eq. (7) PCG solve to
1e-10, E/B update. The chosen form is MIXED32 (int cell + FP32 offset particles, FP32
gather/push/deposit in shared-memory tiles, FP64 field solve with FP32 inner CG); the
plain FP64 GPU path is timed beside it on the same inputs.

--workload scan48 runs the batched parameter scan instead: 48 uneven simulations (grids
128x128 .. 512x256, CFL 0.5-1.0, theta 0.5-0.75, shape orders 1-3, gamma0 = 20, 16 ppc
per species; 87,293,952 particles) in one handle with autotuned tiles; its plain FP64
comparison runs the 48 simulations one after another in their own handles.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload cfg2|cfg1|cfg2q|scan48|cfg5|cfg2x|cfg2n|cfg4]

With N > 1 (launched under torchrun) every rank runs an independent replica with its own
seed (the path has no data-path exchange); value = particles of all ranks x K / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import math
import json
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
    # cfg2's plasma under the explicit FDTD update (Eqs. 3-4) at CFL 0.5
    "cfg2x": (2048, 512, 32, 2, 40.0, 1e-3, 0.5, 0.5, 2),
    # cfg2 with the node-averaged gather reading
    "cfg2n": (2048, 512, 32, 2, 40.0, 1e-3, 1.0, 0.5, 2),
    # config 1's physics on 1024 x 256 with the learned warm start (trained first on
    # 20k (b, dB) pairs of 64 x 64 runs of the same physics), compared with x0 = 0 and
    # the previous step's dB
    "cfg4": (1024, 256, 8, 1, 20.0, 1e-3, 1.0, 0.5, 4),
}
LEARNED = {"cfg4"}
WS_COMPARE = {"cfg2", "cfg4"}  # workloads whose line compares the zero, previous-dB and learned guesses
NET = None  # the trained network of the learned warm start (cfg4)
EXPLICIT = {"cfg2x"}
NODAL = {"cfg2n"}
SHOCK = {
    # the shock configuration: a magnetised pair beam (sigma_B 0.1, Bz with the motional
    # Ey) flowing into the conducting, reflecting wall at x = 0, filling the left half of
    # the box; the moving injector starts at x = nx/2 and feeds the beam behind it
    "cfg5": dict(nx=8192, ny=512, ppc=16, order=3, gamma0=40.0, u_th=1e-3, cfl=1.0, theta=0.501,
                 seed=5, sigma_b=0.1, fill=0.5, inj_seed=105),
}
SCAN = "scan48"
FP32_BYTES_PER_PARTICLE = 48  # 24 B read + 24 B written per MIXED32 particle update
FP32_BYTES_PER_CELL = 36      # 6 FP32 field components read, 3 FP32 currents written
FP64_BYTES_PER_PARTICLE = 80  # 40 B read + 40 B written per FP64 particle update
FP64_BYTES_PER_CELL = 72


def rows_of(name, rank=0):
    """Simulations of a workload as scan-table rows (one row for a single grid)."""
    from paper_1412_2480_gb300 import inputs
    if name == SCAN:
        rows = inputs.scan_table()
        for r in rows:
            r["seed"] += 1000 * rank
        return rows
    if name in SHOCK:
        c = SHOCK[name]
        return [{"k": 0, "nx": c["nx"], "ny": c["ny"], "cfl": c["cfl"], "theta": c["theta"],
                 "order": c["order"], "gamma0": c["gamma0"], "ppc": c["ppc"], "u_th": c["u_th"],
                 "seed": c["seed"] + rank, "walls": True, "sigma_b": c["sigma_b"],
                 "inject_x0": c["fill"] * c["nx"], "inj_seed": c["inj_seed"] + rank}]
    nx, ny, ppc, order, g0, uth, cfl, theta, seed = WORKLOADS[name]
    return [{"k": 0, "nx": nx, "ny": ny, "cfl": cfl, "theta": theta, "order": order,
             "gamma0": g0, "ppc": ppc, "u_th": uth, "seed": seed + rank, "explicit": name in EXPLICIT,
             "nodal": name in NODAL, "learned": name in LEARNED}]


def injected_pairs_per_row(r, n):
    """Pairs per row the moving injector has added after n steps (the schedule pic.h
    defines: floor(ppc (1 + v) cfl n) while the plane is inside the box)."""
    if not r.get("walls"):
        return 0
    v = math.sqrt(1.0 - 1.0 / (r["gamma0"] ** 2))
    width = (1.0 + v) * r["cfl"]
    last = int(math.floor((r["nx"] - r["inject_x0"]) / r["cfl"]))  # steps with injection
    n = min(n, max(0, last))
    return int(math.floor(r["ppc"] * width * n))


def particle_updates(rows, n0, first, k):
    """Particle updates of steps first .. first + k - 1 (n0 particles loaded at step 0)."""
    tot = 0
    for s in range(first, first + k):
        tot += n0 + sum(2 * r["ny"] * injected_pairs_per_row(r, s) for r in rows)
    return tot


def describe(name):
    if name in SHOCK:
        c = SHOCK[name]
        return (f"{c['nx']}x{c['ny']} shock: conducting reflecting wall at x = 0, magnetised pair beam "
                f"(sigma_B {c['sigma_b']}, gamma0 {c['gamma0']:g}, u_th {c['u_th']:g}, {c['ppc']} ppc/species) "
                f"filling x < {c['fill'] * c['nx']:g} and fed by the moving injector, CFL {c['cfl']}, "
                f"theta {c['theta']}, order {c['order']}, PCG rtol 1e-10")
    if name == SCAN:
        rows = rows_of(name)
        cells = sum(r["nx"] * r["ny"] for r in rows)
        return (f"batched scan: 48 periodic simulations, grids 128x128..512x256 ({cells} cells), "
                f"CFL 0.5-1.0, theta 0.5-0.75, orders 1-3, pair plasma gamma0 20, u_th 1e-3, "
                f"16 ppc/species ({2 * 16 * cells} particles), PCG rtol 1e-10, autotuned tiles")
    nx, ny, ppc, order, g0, uth, cfl, theta, seed = WORKLOADS[name]
    if name in EXPLICIT:
        return (f"{nx}x{ny} periodic, explicit FDTD (Eqs. 3-4), CFL {cfl}, order {order}, pair plasma "
                f"gamma0 {g0:g}, u_th {uth:g}, {ppc} ppc/species ({2 * nx * ny * ppc} particles)")
    if name in LEARNED:
        return (f"{nx}x{ny} periodic, CFL {cfl}, theta {theta}, order {order}, pair plasma gamma0 {g0:g}, "
                f"u_th {uth:g}, {ppc} ppc/species ({2 * nx * ny * ppc} particles), PCG rtol 1e-10 from the "
                f"learned warm start (network trained on 20000 (b, dB) pairs of 64x64 runs)")
    if name in NODAL:
        return (f"{nx}x{ny} periodic, node-averaged gather, CFL {cfl}, theta {theta}, order {order}, "
                f"pair plasma gamma0 {g0:g}, u_th {uth:g}, {ppc} ppc/species ({2 * nx * ny * ppc} particles), "
                f"PCG rtol 1e-10")
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
    """nvidia-smi sampling (every 100 ms) while the timed region runs."""

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
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)  # the sampler's first line comes after its start-up
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
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            v = [x.strip() for x in line.split(",")]
            if len(v) < 9:
                continue
            try:
                sm.append(float(v[1]))
                mx.append(float(v[2]))
                pw.append(float(v[3]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if v[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_median": statistics.median(pw) if pw else None}


def traffic_for(kernel_key):
    """Per-launch DRAM bytes of a kernel from the committed ncu summary, only while the
    kernel source is unchanged since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(kernel_key)
    if not d:
        return None
    srcs = d.get("sources") or [d.get("source")]
    return d["bytes_per_launch"] if sources_sha(srcs) == d.get("source_sha") else None


def sources_sha(paths):
    """Hash of the source files a kernel is built from (all of them, in order)."""
    h = hashlib.sha256()
    for rel in paths:
        h.update(open(os.path.join(ROOT, rel), "rb").read())
    return h.hexdigest()[:16]


def make_inputs(rows, pinned=False):
    """Seeded drifting pair plasma of every simulation: a list (per simulation) of two
    species dicts."""
    from paper_1412_2480_gb300 import inputs
    out = []
    for r in rows:
        if r.get("walls"):
            # the beam on [0, inject_x0) (a whole number of cells); its uniform fields
            # (Bz, motional Ey) continue over the rest of the box
            x0 = int(r["inject_x0"])
            w, sp, Fh = inputs.shock_beam(x0, r["ny"], r["ppc"], r["gamma0"], r["u_th"], r["seed"],
                                          sigma_b=r["sigma_b"])
            F = np.empty((6, r["ny"], r["nx"]))
            F[:] = Fh[:, :, -1:]
            F[:, :, :x0] = Fh
            r["fields"] = F
        else:
            w, sp = inputs.drifting_pair_plasma(r["nx"], r["ny"], r["ppc"], r["gamma0"], r["u_th"],
                                                r["seed"])
        if pinned:
            import torch
            pin = []
            for d in sp:
                e = {"qm": d["qm"]}
                for k in ("x", "y", "ux", "uy", "uz"):
                    t = torch.empty(d[k].size, dtype=torch.float64, pin_memory=True)
                    t.numpy()[:] = d[k]
                    e[k] = t.numpy()
                pin.append(e)
            sp = pin
        out.append(sp)
    return out


NO_GRAPH = False  # --no-graph: direct launches (profilers skip kernels of conditional graphs)
NO_COOP = False   # --no-coop: the MIXED32 solve as separate kernels, not one cooperative launch
CG_INNER = False  # --cg-inner: the inner FP32 solve by CG instead of the Chebyshev tiles


def params_of(rows, precision):
    import paper_1412_2480_gb300 as pic
    out = []
    for r in rows:
        kw = {}
        if r.get("walls"):
            kw = dict(bc_x=pic.PIC_BC_WALLS, inject_x0=r["inject_x0"], u_th=r["u_th"], seed=r["inj_seed"])
        flags = (pic.PIC_NO_GRAPH if NO_GRAPH else 0) | (pic.PIC_EXPLICIT if r.get("explicit") else 0)
        flags |= pic.PIC_GATHER_NODAL if r.get("nodal") else 0
        flags |= pic.PIC_NO_COOP if NO_COOP else 0
        flags |= pic.PIC_CG_INNER if CG_INNER else 0
        if r.get("learned") and precision == pic.PIC_MIXED32:
            kw["warm_start"] = pic.PIC_WS_LEARNED
        out.append(pic.pic_params_default(nx=r["nx"], ny=r["ny"], cfl=r["cfl"], theta=r["theta"],
                                          shape_order=r["order"], gamma0=r["gamma0"], ppc=r["ppc"],
                                          precision=precision, cg_rtol=1e-10, cg_max_iter=200,
                                          flags=flags,
                                          tile_x=r.get("tile_x", 0), tile_y=r.get("tile_y", 0), **kw))
    return out


def new_sim(params, stream=None):
    import paper_1412_2480_gb300 as pic
    h = pic.pic_init_batch(params) if len(params) > 1 else pic.pic_init(params[0])
    if stream is not None:
        pic.pic_set_stream(h, stream)
    if any(p.warm_start == pic.PIC_WS_LEARNED for p in params):
        pic.pic_set_cnn(h, NET)
    return h


def train_warm_start(row):
    """The learned warm start of a workload: 20000 (b, dB) pairs from 64 x 64 MIXED32 runs
    of config 1's physics (order 1, 8 ppc per species, gamma0 20) at the workload's CFL and
    theta (the operator of Eq. 7 depends on nothing else), then 3000 training steps on
    the GPU."""
    from paper_1412_2480_gb300 import warmstart
    t0 = time.perf_counter()
    B, X = warmstart.generate_pairs(steps=10000, seeds=(11, 12), cfl=row["cfl"], theta=row["theta"],
                                    order=1, ppc=8, gamma0=20.0, u_th=1e-3)
    t1 = time.perf_counter()
    net, loss, sec = warmstart.train(B, X, iters=3000)
    return net, {"pairs": int(len(B)), "pairs_seconds": t1 - t0, "train_seconds": sec, "train_loss": float(loss)}


def load(h, data, rows=None):
    import paper_1412_2480_gb300 as pic
    for k, sp in enumerate(data):
        pic.pic_select(h, k)
        if rows is not None and rows[k].get("fields") is not None:
            for c in range(6):
                pic.pic_set_fields(h, c, np.ascontiguousarray(rows[k]["fields"][c]).ravel())
        for s, d in enumerate(sp):
            pic.pic_load_particles(h, s, d["x"], d["y"], d["ux"], d["uy"], d["uz"])
    pic.pic_select(h, 0)


def pcg_totals(h, n):
    """(CG iterations, FP64 refinements) the handle's PCG loop has run so far."""
    import paper_1412_2480_gb300 as pic
    m = pic.pic_moments(h)
    return m["loop_iters"], m["loop_refinements"]


def max_over_ranks_of(v, world, device):
    """The largest v over the ranks (the slowest replica's time); v itself on one rank."""
    if world == 1:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(world, updates_per_rank, seconds_max):
    """Whole-job throughput of N independent replicas of the same workload (weak
    scaling): the particle updates of all ranks over the slowest rank's time."""
    return world * updates_per_rank / seconds_max


def run_ours(args, dist):
    import torch

    import paper_1412_2480_gb300 as pic
    rank, world = dist["rank"], dist["world"]
    dev = dist["local_rank"]
    torch.cuda.set_device(dev)
    name = args.workload
    rows = rows_of(name, rank)
    nsim = len(rows)
    ncell = sum(r["nx"] * r["ny"] for r in rows)
    stream = torch.cuda.Stream()
    data = make_inputs(rows, pinned=True)
    npart = sum(d["x"].size for sp in data for d in sp)  # loaded at step 0
    train_info = None
    # the learned warm start: trained for its own workload (cfg4), and for the comparison of
    # the three initial guesses on cfg2 (reported beside the timed form, not timed in it)
    ws_compare = args.precision == "mixed" and nsim == 1 and (
        rows[0].get("learned") or (name in WS_COMPARE and not args.no_ws_compare))
    if ws_compare:
        global NET
        NET, train_info = train_warm_start(rows[0])
    prec = pic.PIC_MIXED32 if args.precision == "mixed" else pic.PIC_FP64
    if nsim > 1 and prec != pic.PIC_MIXED32:
        raise SystemExit("the batched scan runs in MIXED32 (its FP64 comparison is built in)")
    tune = None
    if prec == pic.PIC_MIXED32 and args.tile:
        tx, ty = (int(v) for v in args.tile.lower().split("x"))
        for r in rows:
            r["tile_x"], r["tile_y"] = tx, ty
        tune = {"fixed": args.tile}
    elif prec == pic.PIC_MIXED32:
        # tile shapes per shape order from the autotuner (synthetic scratch batches)
        ps = params_of(rows, prec)
        t0 = time.perf_counter()
        best = pic.pic_autotune_tiles(ps, steps=3)
        for r, p in zip(rows, ps):
            r["tile_x"], r["tile_y"] = p.tile_x, p.tile_y
        tune = {"seconds": time.perf_counter() - t0, "tile_ms_per_order": best,
                "tiles": sorted({(r["order"], r["tile_x"], r["tile_y"]) for r in rows})}
    params = params_of(rows, prec)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def max_over_ranks(v):
        return max_over_ranks_of(v, world, "cuda")

    # ---- end to end through the C ABI with host buffers: load (H2D) + K steps +
    # per-step moments (D2H) + final field readback (D2H) ----
    # warm-up of the load path on a scratch handle, untimed: the first DMA from freshly
    # pinned host pages maps them for the device (several times slower on a host whose
    # memory is fragmented), and the library's temporary pool grows to the load's size
    hw = new_sim(params, stream)
    load(hw, data, rows)
    pic.pic_free(hw)
    h = new_sim(params, stream)
    out_fields = torch.empty(max(r["nx"] * r["ny"] for r in rows), dtype=torch.float64,
                             pin_memory=True).numpy()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    load(h, data, rows)
    t_load = time.perf_counter()
    for _ in range(args.steps):
        pic.pic_step(h, 1)
        pic.pic_moments(h)
    t_steps = time.perf_counter()
    for k, r in enumerate(rows):
        pic.pic_select(h, k)
        for c in range(6):
            pic.pic_fields(h, c, out_fields[: r["nx"] * r["ny"]])
    torch.cuda.synchronize()
    t_end = time.perf_counter()
    e2e_s = max_over_ranks(t_end - t0)
    e2e_parts = {"load_s": t_load - t0, "steps_s": t_steps - t_load, "readback_s": t_end - t_steps}
    barrier()
    h2d = (npart * 5 * 8 + sum(6 * r["nx"] * r["ny"] * 8 for r in rows if r.get("fields") is not None)) / args.steps
    d2h = (6 * ncell * 8) / args.steps + 176
    pic.pic_free(h)

    # ---- device-timed steps with inputs resident ----
    h = new_sim(params, stream)
    load(h, data, rows)
    clocks = Clocks(dev)
    clocks.start()
    pic.pic_step(h, args.warmup)
    it0, ref0 = pcg_totals(h, nsim)
    k0 = pic.pic_moments(h)["kernel_launches"]
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    pic.pic_step(h, args.steps)
    ev1.record(stream)
    ev1.synchronize()
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ms)
    barrier()
    it1, ref1 = pcg_totals(h, nsim)
    m1 = pic.pic_moments(h)
    # Fourier diagnostic of B_z (Sec. 3.1): host-timed pic_spectrum calls on the first
    # simulation, D2H copy of the amplitude map included
    spec = np.empty((rows[0]["ny"], rows[0]["nx"]))
    pic.pic_select(h, 0)
    pic.pic_spectrum(h, pic.PIC_BZ, rows[0]["nx"], rows[0]["ny"])
    t0 = time.perf_counter()
    for _ in range(3):
        spec = pic.pic_spectrum(h, pic.PIC_BZ, rows[0]["nx"], rows[0]["ny"])
    spectrum_ms = (time.perf_counter() - t0) / 3 * 1e3
    n_launch = m1["kernel_launches"] - k0  # counted by the library (step graph's kernel nodes + PCG loop)
    pic.pic_free(h)
    # ---- per-phase CUDA-event timing (one graph per part of the step, events between
    # them) over the same steps as the timed region: a second handle from the same
    # inputs, W warm-up steps, then K profiled steps ----
    h = new_sim(params, stream)
    load(h, data, rows)
    pic.pic_step(h, args.warmup)
    prof = pic.pic_profile(h, args.steps if args.prof_steps <= 0 else args.prof_steps)
    pic.pic_free(h)

    # the three initial guesses of the solve on the same steps (learned warm start only)
    ws_cmp = None
    if train_info is not None:
        ws_cmp = {"training": train_info}
        for nm, ws in (("zero", pic.PIC_WS_ZERO), ("previous_dB", pic.PIC_WS_PREV),
                       ("learned", pic.PIC_WS_LEARNED)):
            ps = params_of(rows, prec)
            for p_ in ps:
                p_.warm_start = ws
            h = new_sim(ps, stream)
            load(h, data, rows)
            pic.pic_step(h, args.warmup)
            pr = pic.pic_profile(h, args.steps)
            ws_cmp[nm] = {"cg_iters_per_step": pr["cg_iters"], "field_solve_ms_per_step": pr["field_ms"],
                          "ms_per_step": pr["step_ms"]}
            pic.pic_free(h)
    res = {"ms": ms_max, "prof": prof, "cg_iters": (it1 - it0) / args.steps,
           "cg_refinements": (ref1 - ref0) / args.steps, "clocks": ck, "launches": n_launch,
           "e2e_s": e2e_s, "e2e_parts": e2e_parts, "h2d": h2d, "d2h": d2h, "npart": npart, "ncell": ncell,
           "updates_timed": particle_updates(rows, npart, args.warmup, args.steps),
           "spectrum_ms": spectrum_ms, "warm_start_comparison": ws_cmp,
           "particles_end": sum(m1["n_particles"]) if nsim == 1 else None,
           "particles_expected": particle_updates(rows, npart, args.warmup + args.steps, 1),
           "updates_e2e": particle_updates(rows, npart, 0, args.steps),
           "rtol_reached": m1["cg_rel_resid"], "tune": tune}

    # ---- plain FP64 GPU path on the same inputs (comparison leg): a single grid, or the
    # scan's simulations one after another in their own handles ----
    if prec == pic.PIC_MIXED32 and not args.skip_fp64 and rank == 0:
        p64 = params_of(rows, pic.PIC_FP64)
        k64 = max(2, args.steps // 8) if nsim == 1 else 2
        tot = field = push = 0.0
        for k in range(nsim):
            h = new_sim([p64[k]], stream)
            load(h, [data[k]], [rows[k]])
            pic.pic_step(h, 2)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pic.pic_step(h, k64)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1) / k64
            prof64 = pic.pic_profile(h, 2)
            field += prof64["field_ms"]
            push += prof64["push_kernel_ms"]
            pic.pic_free(h)
        res["fp64"] = {"ms_per_step": tot,
                       "value": particle_updates(rows, npart, 2, k64) / k64 / (tot * 1e-3),
                       "field_solve_ms_per_step": field, "push_kernel_ms": push, "steps": k64,
                       "how": "one handle" if nsim == 1 else "48 handles one after another"}
    return res


def _patch_sim(name, k):
    """The CPU oracle, as it stands, on patch k of the workload: the same physics on a
    patch of 1/8 of each grid dimension (at least 16 cells) with the same particles per
    cell and its own seed (seed + 1009 k), so that k = 0, 1, ... are independent patches.
    For the scan the patch is its first simulation (128 x 128) whole; for the shock it keeps
    the wall, the beam's fields and the injector at the same fraction of the box."""
    import oracle
    from paper_1412_2480_gb300 import inputs
    r = rows_of(name)[0]
    if name == SCAN:
        sx, sy = r["nx"], r["ny"]
    else:
        sx, sy = max(16, r["nx"] // 8), max(16, r["ny"] // 8)
    seed = r["seed"] + 1009 * k
    F0, inj = None, None
    if r.get("walls"):
        w, sp, F0 = inputs.shock_beam(sx, sy, r["ppc"], r["gamma0"], r["u_th"], seed,
                                      sigma_b=r["sigma_b"])
        x0 = r["inject_x0"] * sx / r["nx"]
        for d in sp:
            keep = d["x"] < x0
            for key in ("x", "y", "ux", "uy", "uz"):
                d[key] = np.ascontiguousarray(d[key][keep])
        inj = dict(x0=x0, ppc=r["ppc"], gamma0=r["gamma0"], u_th=r["u_th"], seed=r["inj_seed"] + k)
    else:
        w, sp = inputs.drifting_pair_plasma(sx, sy, r["ppc"], r["gamma0"], r["u_th"], seed)
    species = [oracle.Species(d["qm"], w, d["x"], d["y"], d["ux"], d["uy"], d["uz"]) for d in sp]
    sim = oracle.OracleSim(sx, sy, r["cfl"], r["theta"], r["order"], species, cg_rtol=1e-10,
                           fields=F0, walls=bool(r.get("walls")), injector=inj,
                           solver="explicit" if r.get("explicit") else "implicit",
                           gather="nodal" if r.get("nodal") else "staggered")
    kind = "patch" if name != SCAN else "simulation"
    what = (f"{sx}x{sy} {kind} (order {r['order']}, {r['ppc']} ppc/species, gamma0 {r['gamma0']:g}"
            f"{', walls and injector' if r.get('walls') else ''})")
    return sim, what


def _oracle_worker(name, k, conn):
    """One host process stepping one oracle patch on command (single-threaded oracle)."""
    sim, what = _patch_sim(name, k)
    conn.send((sum(s.n for s in sim.species), what))
    while conn.recv() is not None:
        n = sum(s.n for s in sim.species)
        sim.step(1)
        conn.send(n)


class OraclePatches:
    """`cores` independent oracle processes, one patch each, stepped together: a step's
    particle updates are the sum over the patches, its time the wall time until the
    slowest patch has finished. Processes are spawned (never forked after a GPU call)."""

    def __init__(self, name, cores):
        import multiprocessing as mp
        import oracle
        oracle.build()  # once, before the workers load it
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for k in range(cores):
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_oracle_worker, args=(name, k, b), daemon=True)
            pr.start()
            self.conns.append(a)
            self.procs.append(pr)
        ready = [c.recv() for c in self.conns]
        self.particles = sum(n for n, _ in ready)
        self.what = ready[0][1]
        self.cores = cores

    def step(self):
        t0 = time.perf_counter()
        for c in self.conns:
            c.send(1)
        n = sum(c.recv() for c in self.conns)
        return n, time.perf_counter() - t0

    def close(self):
        for c in self.conns:
            c.send(None)
        for pr in self.procs:
            pr.join(timeout=30)


def _timed_patches(name, cores, seconds, max_steps=50):
    P = OraclePatches(name, cores)
    try:
        P.step()  # warm-up
        upd, wall, steps = 0, 0.0, 0
        while (wall < seconds or steps < 2) and steps < max_steps:
            n, t = P.step()
            upd += n
            wall += t
            steps += 1
    finally:
        P.close()
    return upd, wall, steps, P.what


def oracle_sample(name, seconds_target=10.0):
    """The CPU oracle as it stands on the machine's host cores: os.cpu_count() independent
    single-threaded processes, one patch each (aggregate particle updates/s), and one
    process alone beside it (one core)."""
    cores = os.cpu_count() or 1
    upd, wall, steps, what = _timed_patches(name, cores, seconds_target)
    upd1, wall1, steps1, _ = _timed_patches(name, 1, seconds_target / 2)
    return {"value": upd / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes, each one {what} with its own seed ({upd // (steps * cores)} "
                      f"particles each), {steps} whole steps in {wall:.1f} s of wall time on {cores} host cores",
            "single_core": {"value": upd1 / wall1, "unit": UNIT, "cores": 1,
                            "sample": f"one {what} process, {steps1} whole steps in {wall1:.1f} s"}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + sorted(SHOCK) + [SCAN], default="cfg2")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--prof-steps", type=int, default=0,
                    help="steps of per-phase timing (0: the timed steps again, from the same start)")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--tile", default="", help="fixed MIXED32 tile TXxTY instead of the autotuner's choice")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ws-compare", action="store_true",
                    help="skip the comparison of the solve's initial guesses (zero, previous dB, learned)")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch kernels directly (for profiler launch lists), not a bench number")
    ap.add_argument("--no-coop", action="store_true",
                    help="run the MIXED32 solve as separate kernels (the comparison path)")
    ap.add_argument("--cg-inner", action="store_true",
                    help="MIXED32 inner solve by CG instead of the Chebyshev tiles (the comparison path)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    global NO_GRAPH, NO_COOP, CG_INNER
    NO_GRAPH = args.no_graph
    NO_COOP = args.no_coop
    CG_INNER = args.cg_inner

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    dist = {"world": world, "rank": rank, "local_rank": local_rank}
    rows = rows_of(args.workload)
    npart = sum(2 * r["ppc"] * int(r.get("inject_x0", r["nx"])) * r["ny"] for r in rows)

    if args.impl == "reference":
        if rank != 0:
            return
        # The oracle is the reference arm: every step is one whole step of os.cpu_count()
        # independent patches of the workload, one single-threaded oracle process each, on
        # the machine's host cores; the line reports what was run (the patches), not an
        # extrapolation to the full workload.
        cores = os.cpu_count() or 1
        P = OraclePatches(args.workload, cores)
        try:
            for _ in range(args.warmup):
                P.step()
            per = [P.step() for _ in range(args.steps)]
        finally:
            P.close()
        upd = sum(n for n, _ in per)
        wall = sum(t for _, t in per)
        v = upd / wall
        ms = statistics.median(t for _, t in per) * 1e3
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{cores} processes, each one {P.what} ({P.particles} particles in all), "
                         f"{args.steps} timed whole steps in {wall:.1f} s"}
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"{cores} independent copies (own seeds) of a {P.what} "
                                       f"cut from the workload: {describe(args.workload)}",
                           "particles_per_step": P.particles, "l2": "n/a (host)"},
                "cpu_baseline": cpu,
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    res = run_ours(args, dist)
    if rank != 0:
        return
    # the host-side oracle sample runs after the GPU legs: its processes would otherwise
    # still load the host cores that the end-to-end leg's calls run on
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(args.workload)
    value = job_value(world, res["updates_timed"], res["ms"] * 1e-3)
    npart = res["updates_timed"] / args.steps  # particles per step, averaged over the timed steps
    hbm, src = peaks()
    mixed = args.precision == "mixed"
    bpp = FP32_BYTES_PER_PARTICLE if mixed else FP64_BYTES_PER_PARTICLE
    bpc = FP32_BYTES_PER_CELL if mixed else FP64_BYTES_PER_CELL
    alg_bytes = int(bpp * npart + bpc * res["ncell"])
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
                   "form": ("MIXED32 (int cell + FP32 offset; FP32 gather/push/deposit; "
                            + ("FP64 explicit field update)" if args.workload in EXPLICIT else
                               "FP64 field update and PCG residual with FP32 inner CG)")
                            + (", solve as separate kernels" if NO_COOP else "")
                            + (", inner CG" if CG_INNER or NO_COOP else ", inner Chebyshev tiles")) if mixed else "FP64",
                   "l2": "inputs larger than L2 (particle state 1.6 GB MIXED32 / 2.7 GB FP64 for cfg2, "
                         "2.1 GB for scan48)",
                   "replicas": world},
        "field_solve_ms_per_step": res["prof"]["field_ms"],
        "particle_ms_per_step": res["prof"]["particle_ms"],
        "cg_iters_per_step": res["cg_iters"],
        "cg_refinements_per_step": res["cg_refinements"],
        "e2e": {"value": job_value(world, res["updates_e2e"], res["e2e_s"]), "unit": UNIT,
                "h2d_bytes_per_step": int(res["h2d"]), "d2h_bytes_per_step": int(res["d2h"]),
                "what": "pic_load_particles from pinned host arrays + K x (pic_step(1) + pic_moments) "
                        "+ pic_fields x 6 per simulation",
                "seconds": {k: round(v, 4) for k, v in res["e2e_parts"].items()}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic, "kernel": key,
                     "peak_source": src,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "kernel_ms": kms},
        "gpu_launches": res["launches"],
        "particles_end": {"counted": res["particles_end"], "schedule": res["particles_expected"]},
        "spectrum_ms": res["spectrum_ms"],
        **({"warm_start_comparison": res["warm_start_comparison"]} if res.get("warm_start_comparison") else {}),
        "clocks": res["clocks"],
    }
    if res["tune"]:
        line["autotune"] = res["tune"]
    if "fp64" in res:
        line["plain_fp64"] = res["fp64"]
        line["speedup_vs_plain_fp64"] = res["fp64"]["ms_per_step"] / (res["ms"] / args.steps)
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
