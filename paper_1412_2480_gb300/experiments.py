"""Parameter scans of numerical Cherenkov growth (Sec. 3) on the GPU, through the C ABI.

A run is the paper's test of Sec. 3: a periodic 128 x 128 box, an electron-positron flow
of Lorentz factor 100 along x with a 10% rest-frame thermal spread, 100 particles per
cell per species, fields starting at zero. The growth rate of the instability is the
largest slope of ln U_B(t) over a sliding window (least squares), in units of c/dx.

    python -m paper_1412_2480_gb300.experiments theta-scan [--steps 5000] [--ppc 100]

prints one JSON object: growth rates for theta in {0.5, 0.501, 0.502, 0.503}, shape
orders 1 and 2, at CFL 1 (the slowly growing mode of Sec. 3.3), for the staggered gather
and for the node-averaged reading (PIC_GATHER_NODAL).
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


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("what", choices=["theta-scan"])
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--ppc", type=int, default=100)
    ap.add_argument("--cfl", type=float, default=1.0)
    args = ap.parse_args()
    if not math.isfinite(args.cfl) or not 0 < args.cfl <= 1:
        raise SystemExit("cfl must lie in (0, 1]")
    print(json.dumps(theta_scan(steps=args.steps, ppc=args.ppc, cfl=args.cfl)))


if __name__ == "__main__":
    main()
