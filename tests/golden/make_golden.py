"""Writes tests/golden/vacuum_te_cfl05.txt by running the CPU oracle only.

The table is the Fig. 2 setting of the paper (Sec. 2: c dt/dx = c dt/dy = 0.5) on a
32 x 32 periodic grid: for each mode (mx, my) and theta, a standing TE wave
Bz = cos(k.x), E = 0 is advanced 8 steps and the Bz amplitude after each step is
recorded (projection on the initial mode). The test suite compares the table with the
paper's dispersion relation, Eq. (15) at theta = 1/2 and Eq. (10) otherwise.

Run from the repository root:  python tests/golden/make_golden.py
"""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402

NX = NY = 32
CFL = 0.5
THETAS = (0.5, 0.501)
MODES = [(1, 0), (0, 1), (2, 3), (5, 5), (8, 0), (12, 4), (16, 16), (3, 14)]
STEPS = 8


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "vacuum_te_cfl05.txt")
    jj, ii = np.meshgrid(np.arange(NY), np.arange(NX), indexing="ij")
    lines = ["# written by tests/golden/make_golden.py (CPU oracle only); Fig. 2 setting of Sec. 2",
             "# theta mx my a_1 ... a_8   (Bz amplitude after n steps, initial amplitude 1)"]
    for theta in THETAS:
        for mx, my in MODES:
            kx, ky = 2 * math.pi * mx / NX, 2 * math.pi * my / NY
            mode = np.cos(kx * (ii + 0.5) + ky * (jj + 0.5))
            F = np.zeros((6, NY, NX))
            F[5] = mode
            sim = oracle.OracleSim(NX, NY, CFL, theta, 2, [], cg_rtol=1e-15, fields=F)
            amps = []
            for _ in range(STEPS):
                sim.step()
                amps.append(float(np.sum(sim.fields()[5] * mode) / np.sum(mode * mode)))
            lines.append(f"{theta:.3f} {mx} {my} " + " ".join(f"{a:.15e}" for a in amps))
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
