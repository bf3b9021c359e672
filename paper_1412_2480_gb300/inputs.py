"""Seeded synthetic inputs: relativistic drifting electron-positron pair plasmas
shaped like the runs of Ikeya & Matsumoto (PASJ 2015, Sec. 3 and Sec. 4).

This module holds none of the particle cycle's arithmetic; it only builds initial
states. Both the CUDA path (tests, benchmark) and the CPU oracle read the same arrays
from it, so the two start from bit-identical inputs.

Recipe (all in code units: c = 1, lengths in units of the cell size dx = dy = 1 by
default):
  * ppc macro-particles per cell per species, positions uniform-random inside their
    cell, generated cell by cell in storage order (j major, i minor);
  * co-located pairs: every positron sits on the position of one electron, so the
    charge density and E vanish at t = 0 (the paper starts from E = B = 0, Sec. 3);
  * momenta: rest-frame Gaussian with standard deviation u_th per component (units of
    c), Lorentz-boosted to the drift Lorentz factor gamma0 along +x, drawn
    independently for each species;
  * macro weight w from the plasma frequency in the flow frame (Sec. 4 definition)
    omega_pe^2 = 4 pi n q^2 / (m gamma0), with n = ppc / (dx dy) per species and
    q = m = w per macro-particle, so w = omega_pe^2 gamma0 dx dy / (4 pi ppc) and
    omega_pe = c / skin_depth.
"""
from __future__ import annotations

import math

import numpy as np

POSITRON, ELECTRON = 0, 1
QM = (+1.0, -1.0)  # charge-to-mass ratio (sign) of each species, in units of e/m_e


def macro_weight(ppc: int, gamma0: float, skin_depth: float = 10.0, dx: float = 1.0,
                 dy: float = 1.0) -> float:
    wpe = 1.0 / skin_depth
    return wpe * wpe * gamma0 * dx * dy / (4.0 * math.pi * ppc)


def boosted_momenta(rng: np.random.Generator, n: int, gamma0: float, u_th: float):
    """Rest-frame Gaussian momenta boosted along +x (u = gamma v, c = 1)."""
    up = rng.standard_normal((3, n)) * u_th
    gp = np.sqrt(1.0 + up[0] ** 2 + up[1] ** 2 + up[2] ** 2)
    beta0 = math.sqrt(max(0.0, 1.0 - 1.0 / (gamma0 * gamma0)))
    ux = gamma0 * (up[0] + beta0 * gp)
    return ux, up[1].copy(), up[2].copy()


def drifting_pair_plasma(nx: int, ny: int, ppc: int, gamma0: float, u_th: float, seed: int,
                         dx: float = 1.0, dy: float = 1.0, skin_depth: float = 10.0,
                         colocated: bool = True):
    """Returns (w, [species0, species1]); each species is a dict with keys
    qm, x, y, ux, uy, uz (float64 arrays of nx*ny*ppc entries)."""
    rng = np.random.Generator(np.random.Philox(int(seed)))
    n = nx * ny * ppc
    cell = np.repeat(np.arange(nx * ny, dtype=np.int64), ppc)
    ci = (cell % nx).astype(np.float64)
    cj = (cell // nx).astype(np.float64)
    del cell
    x = (ci + rng.random(n)) * dx
    y = (cj + rng.random(n)) * dy
    del ci, cj
    out = []
    for s in (POSITRON, ELECTRON):
        if s == ELECTRON and not colocated:
            x = (np.repeat(np.arange(nx * ny) % nx, ppc) + rng.random(n)) * dx
            y = (np.repeat(np.arange(nx * ny) // nx, ppc) + rng.random(n)) * dy
        ux, uy, uz = boosted_momenta(rng, n, gamma0, u_th)
        out.append({"qm": QM[s], "x": x, "y": y, "ux": ux, "uy": uy, "uz": uz})
    return macro_weight(ppc, gamma0, skin_depth, dx, dy), out


def random_fields(nx: int, ny: int, amplitude: float, seed: int) -> np.ndarray:
    """Smooth seeded field state (6, ny, nx): a few random Fourier modes per component,
    used to exercise the gather and push with nonzero E and B."""
    rng = np.random.Generator(np.random.Philox(int(seed) + 7919))
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    F = np.zeros((6, ny, nx))
    for c in range(6):
        for _ in range(4):
            mx, my = rng.integers(-4, 5), rng.integers(-4, 5)
            ph = rng.random() * 2 * math.pi
            F[c] += rng.standard_normal() * np.cos(2 * math.pi * (mx * ii / nx + my * jj / ny) + ph)
    return F * amplitude


# ---- the batched parameter scan: 48 uneven simulations ------------------------------
# The paper scans the CFL number (Sec. 3.2), theta and the shape order (Sec. 3.3); the
# scan table crosses those values with uneven grid sizes. Row k: CFL = SCAN_CFL[k mod 6],
# theta = SCAN_THETA[floor(k/6) mod 4], shape order 1 + (k + floor(k/24)) mod 3, grid
# SCAN_GRIDS[5k mod 8], gamma0 = 20, 16 particles per cell per species, 1e-3 spread,
# seed 3 + k. The committed copy is scan48.json beside this module.
SCAN_CFL = (0.5, 0.6, 0.7, 0.8, 0.9, 1.0)
SCAN_THETA = (0.5, 0.55, 0.6, 0.75)
SCAN_GRIDS = ((128, 128), (192, 128), (256, 128), (192, 192), (256, 192), (256, 256),
              (384, 256), (512, 256))


def scan_table(n: int = 48) -> list:
    rows = []
    for k in range(n):
        nx, ny = SCAN_GRIDS[(5 * k) % len(SCAN_GRIDS)]
        rows.append({"k": k, "nx": nx, "ny": ny, "cfl": SCAN_CFL[k % 6],
                     "theta": SCAN_THETA[(k // 6) % 4], "order": 1 + (k + k // 24) % 3,
                     "gamma0": 20.0, "ppc": 16, "u_th": 1e-3, "seed": 3 + k})
    return rows


# ---- the shock configuration: a magnetised pair beam flowing into a reflecting wall ----
def shock_beam(nx: int, ny: int, ppc: int, gamma0: float, u_th: float, seed: int,
               sigma_b: float = 0.1, dx: float = 1.0, dy: float = 1.0, skin_depth: float = 10.0):
    """Co-located pairs filling [0, nx dx) x [0, ny dy), drifting toward the wall at
    x = 0 with Lorentz factor gamma0 (the paper's shock set-up mirrored: it injects at
    the left and reflects at the right, Sec. 4), in a uniform out-of-plane field Bz = B0
    of magnetisation sigma_b = B0^2 / (4 pi gamma0 n m c^2) (n: both species) and the
    motional field Ey = -v B0 that lets the beam drift undeflected (zero on the wall
    column). Returns (macro weight, species list, fields (6, ny, nx))."""
    w, sp = drifting_pair_plasma(nx, ny, ppc, gamma0, u_th, seed, dx=dx, dy=dy,
                                 skin_depth=skin_depth)
    for d in sp:
        d["ux"] = -d["ux"]
    wpe = 1.0 / skin_depth
    # n m c^2 over both species = 2 ppc w / (dx dy) = omega_pe^2 gamma0 / (2 pi)
    b0 = math.sqrt(sigma_b * 4.0 * math.pi * gamma0 * 2.0 * ppc * w / (dx * dy))
    v = math.sqrt(1.0 - 1.0 / (gamma0 * gamma0))
    F = np.zeros((6, ny, nx))
    F[5] = b0
    F[1] = -v * b0
    F[1][:, 0] = 0.0
    return w, sp, F
