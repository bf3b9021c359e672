"""Writes tests/golden/shock_noise_reduced.json by running the CPU oracle only.

Config 5 (the relativistic shock of Sec. 4) at reduced size: 1024 x 128 cells, a
conducting reflecting wall at x = 0, a magnetised pair beam (sigma_B = 0.1 in Bz with
the motional Ey, gamma0 = 40, 1e-3 spread, 16 particles per cell per species) filling
x < 512 and flowing toward the wall, fed by the moving injector that starts at x = 512;
CFL 1, theta = 0.501, shape order 3. 400 steps (omega_pe t = 40 at c/omega_pe = 10
cells): the reflected beam builds the shock at the wall while the beam ahead of it, the
upstream, carries the numerical noise the paper measures.

Recorded per step: the upstream magnetic noise energy, sum over the cells with
256 <= x < 512 of |B - B0 z|^2 dx dy / (8 pi) (B0 the initial uniform field; that band
holds upstream beam throughout: the shock front stays below x = 256 within 400 steps and
the band fills from the injector behind it), the total field energies U_E and U_B, the
particle count, and the SHA-256 of the seeded initial particles.

Run from the repository root:  python tests/golden/make_shock_noise.py   (about an hour)
"""
import hashlib
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

NX, NY, PPC, ORDER, GAMMA0, UTH, CFL, THETA = 1024, 128, 16, 3, 40.0, 1e-3, 1.0, 0.501
SIGMA_B, SEED, INJ_SEED = 0.1, 5, 105
X0 = NX // 2
BAND = (NX // 4, NX // 2)
STEPS = 400


def setup():
    from paper_1412_2480_gb300 import inputs
    w, sp, F0 = inputs.shock_beam(NX, NY, PPC, GAMMA0, UTH, SEED, sigma_b=SIGMA_B)
    for d in sp:
        keep = d["x"] < X0
        for k in ("x", "y", "ux", "uy", "uz"):
            d[k] = np.ascontiguousarray(d[k][keep])
    inj = dict(x0=float(X0), ppc=PPC, gamma0=GAMMA0, u_th=UTH, seed=INJ_SEED)
    return w, sp, F0, inj


def input_hash(sp):
    h = hashlib.sha256()
    for d in sp:
        for k in ("x", "y", "ux", "uy", "uz"):
            h.update(np.ascontiguousarray(d[k], dtype=np.float64).tobytes())
    return h.hexdigest()


def band_noise(F, b0):
    """Upstream magnetic noise energy: |B - B0 z|^2 / (8 pi) summed over the band."""
    F = F.reshape(6, NY, NX)
    sl = slice(*BAND)
    return float((F[3][:, sl] ** 2 + F[4][:, sl] ** 2 + (F[5][:, sl] - b0) ** 2).sum() / (8 * math.pi))


def main():
    import oracle
    oracle.build()
    w, sp, F0, inj = setup()
    b0 = float(F0[5][0, 0])
    species = [oracle.Species(d["qm"], w, d["x"], d["y"], d["ux"], d["uy"], d["uz"]) for d in sp]
    sim = oracle.OracleSim(NX, NY, CFL, THETA, ORDER, species, cg_rtol=1e-10, fields=F0, walls=True,
                           injector=inj)
    noise, ue, ub, npart = [], [], [], []
    for n in range(STEPS):
        sim.step(1)
        F = sim.fields()
        noise.append(band_noise(F, b0))
        e, b = sim.energies()[:2]
        ue.append(float(e))
        ub.append(float(b))
        npart.append(int(sim.species[0].n))
        if n % 20 == 0:
            print(n, noise[-1], flush=True)
    out = {"written_by": "tests/golden/make_shock_noise.py (CPU oracle only)",
           "workload": {"nx": NX, "ny": NY, "ppc": PPC, "order": ORDER, "gamma0": GAMMA0, "u_th": UTH,
                        "cfl": CFL, "theta": THETA, "sigma_b": SIGMA_B, "seed": SEED,
                        "inject_x0": X0, "inject_seed": INJ_SEED, "band": list(BAND), "steps": STEPS,
                        "cg_rtol": 1e-10},
           "input_sha256": input_hash(sp), "b0": b0,
           "after_step": {"band_noise": [float(f"{v:.10e}") for v in noise],
                          "U_E": [float(f"{v:.10e}") for v in ue], "U_B": [float(f"{v:.10e}") for v in ub],
                          "n_per_species": npart}}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "shock_noise_reduced.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
