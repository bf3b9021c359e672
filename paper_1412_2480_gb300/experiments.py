"""Parameter scans of numerical Cherenkov growth (Sec. 3) on the GPU, through the C ABI.

A run is the paper's test of Sec. 3: a periodic 128 x 128 box, an electron-positron flow
of Lorentz factor 100 along x with a 10% rest-frame thermal spread, 100 particles per
cell per species, fields starting at zero. The growth rate of the instability is the
largest slope of ln U_B(t) over a sliding window (least squares), in units of c/dx.

    python -m paper_1412_2480_gb300.experiments theta-scan [--steps 5000] [--ppc 100]

prints one JSON object: growth rates for theta in {0.5, 0.501, 0.502, 0.503}, shape
orders 1 and 2, at CFL 1 (the slowly growing mode of Sec. 3.3), for the staggered gather
and for the node-averaged reading (PIC_GATHER_NODAL).

    python -m paper_1412_2480_gb300.experiments shock --cfl 1.0 [--nx 5650 --ny 990]

runs the relativistic shock of Sec. 4 (5650 x 990 cells, Gamma = 100, 5% thermal
spread, 50 particles per cell per species, order 2, theta = 0.501, no background field:
a Weibel-mediated shock) to omega_pe t = 177, mirrored as the wall and injector of
include/pic.h set it up (wall at x = 0, the flow moving in -x), and prints the
transversely averaged electron density n_e(x)/n_0 and magnetic energy density
B_z^2/8pi over the upstream kinetic energy density, with the shock position, the
density jump and the upstream and peak magnetic energy fractions.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import inputs


def run_history(cfl=1.0, theta=0.501, order=2, steps=5000, every=50, nx=128, ny=128, ppc=100,
                gamma0=100.0, u_th=0.1, seed=7, flags=0):
    """U_B, U_E, U_K every `every` steps of the Sec. 3 test (MIXED32)."""
    from . import (PIC_MIXED32, pic_free, pic_init, pic_load_particles, pic_moments,
                   pic_params_default, pic_step)
    w, sp = inputs.drifting_pair_plasma(nx, ny, ppc, gamma0, u_th, seed)
    prm = pic_params_default(nx=nx, ny=ny, cfl=cfl, theta=theta, shape_order=order, gamma0=gamma0,
                             ppc=ppc, precision=PIC_MIXED32, cg_rtol=1e-8, flags=flags)
    h = pic_init(prm)
    hist = []
    try:
        for s, d in enumerate(sp):
            pic_load_particles(h, s, d["x"], d["y"], d["ux"], d["uy"], d["uz"])
        for _ in range(steps // every):
            pic_step(h, every)
            m = pic_moments(h)
            hist.append((m["step"] * cfl, m["U_B"], m["U_E"], m["U_K"]))
    finally:
        pic_free(h)
    return np.array(hist)


def growth_rate(hist, window=1000.0):
    """Largest least-squares slope of ln U_B over a window of `window` time units."""
    t, ub = hist[:, 0], hist[:, 1]
    good = ub > 0
    t, lu = t[good], np.log(ub[good])
    best = 0.0
    for a in range(len(t)):
        b = np.searchsorted(t, t[a] + window)
        if b - a < 4:
            break
        slope = np.polyfit(t[a:b], lu[a:b], 1)[0]
        best = max(best, slope)
    return best


def theta_scan(steps=5000, ppc=100, cfl=1.0, thetas=(0.5, 0.501, 0.502, 0.503), orders=(1, 2)):
    from . import PIC_GATHER_NODAL
    out = {"cfl": cfl, "steps": steps, "ppc": ppc, "rates": []}
    for gather, flags in (("staggered", 0), ("nodal", PIC_GATHER_NODAL)):
        for order in orders:
            for theta in thetas:
                t0 = time.perf_counter()
                h = run_history(cfl=cfl, theta=theta, order=order, steps=steps, ppc=ppc, flags=flags)
                out["rates"].append({"gather": gather, "order": order, "theta": theta,
                                     "growth_rate": growth_rate(h),
                                     "U_B_over_U_K_end": float(h[-1, 1] / h[-1, 3]),
                                     "seconds": time.perf_counter() - t0})
    return out


def shock_run(cfl=1.0, nx=5650, ny=990, ppc=50, gamma0=100.0, u_th=0.05, t_end=177.0,
              skin_depth=10.0, theta=0.501, order=2, seed=11, every=50, stride=10):
    """The Sec. 4 shock, mirrored: wall at x = 0, the flow moving in -x, the moving
    injector (include/pic.h) feeding it from x0 so that its plane reaches the far end of
    the box at omega_pe t = t_end. Lengths in cells (c/omega_pe = skin_depth cells)."""
    from . import (PIC_BC_WALLS, PIC_BZ, PIC_DENSITY_E, PIC_MIXED32, fields_numpy, pic_free, pic_init,
                   pic_load_particles, pic_moments, pic_params_default, pic_step)
    steps = int(round(t_end * skin_depth / cfl))
    x0 = int(math.floor(nx - steps * cfl - 1))
    if x0 < 2 * cfl + 1:
        raise ValueError("the box is too short for the run: the injector needs nx > t_end * skin_depth")
    t0 = time.perf_counter()
    w, sp, _ = inputs.shock_beam(x0, ny, ppc, gamma0, u_th, seed, sigma_b=0.0, skin_depth=skin_depth)
    prm = pic_params_default(nx=nx, ny=ny, cfl=cfl, theta=theta, shape_order=order, gamma0=gamma0,
                             ppc=ppc, skin_depth=skin_depth, precision=PIC_MIXED32, cg_rtol=1e-8,
                             bc_x=PIC_BC_WALLS, inject_x0=float(x0), u_th=u_th, seed=seed + 1000)
    h = pic_init(prm)
    hist = []
    try:
        for s, d in enumerate(sp):
            pic_load_particles(h, s, d["x"], d["y"], d["ux"], d["uy"], d["uz"])
        del sp
        t_load = time.perf_counter() - t0
        t1 = time.perf_counter()
        done = 0
        while done < steps:
            k = min(every, steps - done)
            pic_step(h, k)
            done += k
            m = pic_moments(h)
            hist.append((m["step"] * cfl / skin_depth, m["U_B"], m["U_E"], m["U_K"],
                         m["n_particles"][0] + m["n_particles"][1]))
        t_run = time.perf_counter() - t1
        ne = fields_numpy(h, PIC_DENSITY_E, nx, ny)
        bz = fields_numpy(h, PIC_BZ, nx, ny)
    finally:
        pic_free(h)
    n0 = ppc  # upstream electrons per unit area (dx = dy = 1)
    ne_x = ne.mean(axis=0) / n0
    eb_x = (bz * bz).mean(axis=0) / (8 * math.pi)
    ek_up = 2.0 * (gamma0 - 1.0) * w * ppc  # both species, per unit area
    eps_b = eb_x / ek_up
    # shock front: the upstream-most x (largest, the flow comes from +x) where the
    # density, smoothed over a skin depth, exceeds twice the upstream value
    k = max(1, int(skin_depth))
    smooth = np.convolve(ne_x, np.ones(k) / k, mode="same")
    above = np.nonzero(smooth[: x0] > 2.0)[0]
    xs = int(above.max()) if above.size else 0
    down = ne_x[int(0.2 * xs): int(0.8 * xs)] if xs > 10 else ne_x[:0]
    up_lo, up_hi = xs + int(20 * skin_depth), min(nx - int(20 * skin_depth), xs + int(80 * skin_depth))
    up = eps_b[up_lo:up_hi] if up_hi > up_lo else eps_b[:0]
    return {"cfl": cfl, "nx": nx, "ny": ny, "ppc": ppc, "steps": steps, "omega_pe_t": steps * cfl / skin_depth,
            "particles_end": int(hist[-1][4]), "seconds_load": t_load, "seconds_run": t_run,
            "ms_per_step": t_run / steps * 1e3,
            "shock_x_cells": xs, "shock_x_skin_depths": xs / skin_depth,
            "shock_speed_c": xs / (steps * cfl) if xs else 0.0,
            "downstream_density_ratio": float(down.mean()) if down.size else None,
            "upstream_eps_b": float(up.mean()) if up.size else None,
            "peak_eps_b": float(eps_b.max()), "peak_eps_b_x_cells": int(eps_b.argmax()),
            "history": [list(map(float, r)) for r in hist],
            "profile_x_cells": list(range(0, nx, stride)),
            "profile_ne_over_n0": [float(v) for v in ne_x[::stride]],
            "profile_eps_b": [float(v) for v in eps_b[::stride]]}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("what", choices=["theta-scan", "shock"])
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--ppc", type=int, default=None)
    ap.add_argument("--cfl", type=float, default=1.0)
    ap.add_argument("--nx", type=int, default=5650)
    ap.add_argument("--ny", type=int, default=990)
    ap.add_argument("--t-end", type=float, default=177.0)
    args = ap.parse_args()
    if not math.isfinite(args.cfl) or not 0 < args.cfl <= 1:
        raise SystemExit("cfl must lie in (0, 1]")
    if args.what == "theta-scan":
        print(json.dumps(theta_scan(steps=args.steps, ppc=args.ppc or 100, cfl=args.cfl)))
    else:
        print(json.dumps(shock_run(cfl=args.cfl, nx=args.nx, ny=args.ny, ppc=args.ppc or 50,
                                   t_end=args.t_end)))


if __name__ == "__main__":
    main()
