"""Edge and degenerate cases of the particle cycle, GPU against the oracle or a closed
form: rectangular cells (dx != dy), the backward-Euler end of the implicitness range
(theta = 1), particles sitting exactly on cell and half-cell boundaries (the shape
tie-breaks), and long thin grids (one tile high or wide, ragged in both directions)."""
import math

import numpy as np
import pytest

import oracle
import paper_1412_2480_gb300 as pic
from closed_forms import amplification
from paper_1412_2480_gb300 import inputs
from runners import check, match_particles, rel, run_gpu

pytestmark = pytest.mark.gpu
TOL32 = 2e-5


def oracle_run(nx, ny, w, sp, F0, steps, order, cfl, dx=1.0, dy=1.0, theta=0.5):
    species = [oracle.Species(d["qm"], w, d["x"], d["y"], d["ux"], d["uy"], d["uz"]) for d in sp]
    sim = oracle.OracleSim(nx, ny, cfl, theta, order, species, dx=dx, dy=dy, cg_rtol=1e-13, fields=F0)
    sim.step(steps)
    F = np.concatenate([sim.fields(), sim.J.reshape(3, ny, nx)])
    return F, [np.stack([s.x, s.y, s.ux, s.uy, s.uz]) for s in sim.species]


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_MIXED32])
def test_rectangular_cells_match_oracle(precision, order):
    nx, ny, ppc, dx, dy, cfl = 48, 32, 3, 1.0, 0.5, 0.4  # dt = 0.4 dx < dy
    w, sp = inputs.drifting_pair_plasma(nx, ny, ppc, 3.0, 0.3, seed=160 + order, dx=dx, dy=dy,
                                        colocated=False)
    F0 = inputs.random_fields(nx, ny, 0.05, seed=161)
    kw = {"tile_x": 16, "tile_y": 8} if precision == pic.PIC_MIXED32 else {}
    Fg, pg, _ = run_gpu(nx, ny, ppc, sp, F0, 2, order, cfl=cfl, gamma0=3.0, cg_rtol=1e-13,
                        precision=precision, dx=dx, dy=dy, **kw)
    Fo, po = oracle_run(nx, ny, w, sp, F0, 2, order, cfl, dx=dx, dy=dy)
    tol = 1e-12 if precision == pic.PIC_FP64 else TOL32
    for c in range(9):
        check(Fg[c], Fo[c], tol, f"quantity {c}")
    for s in range(2):
        d = match_particles(pg[s], po[s], [nx * dx, ny * dy, 3.0, 3.0, 3.0])
        assert d < (1e-12 if precision == pic.PIC_FP64 else 1e-5), d


@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_MIXED32])
def test_backward_euler_vacuum_mode(precision):
    # theta = 1: the mode decays by the exact amplification of Eq. (10) every step
    nx, ny, theta, cfl, mx, my = 48, 32, 1.0, 1.0, 5, 3
    kx, ky = 2 * math.pi * mx / nx, 2 * math.pi * my / ny
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    F0 = np.zeros((6, ny, nx))
    F0[5] = np.cos(kx * (ii + 0.5) + ky * (jj + 0.5))
    lam = amplification(theta, cfl * math.hypot(math.sin(kx / 2), math.sin(ky / 2)))
    assert abs(lam) < 0.99  # backward Euler damps the mode
    for n in (1, 5):
        Fg, _, _ = run_gpu(nx, ny, 1, [], F0, n, 2, cfl=cfl, theta=theta, cg_rtol=1e-13,
                           precision=precision, want_particles=False)
        np.testing.assert_allclose(Fg[5], (lam ** n).real * F0[5], rtol=0, atol=1e-12)


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_MIXED32])
def test_particles_on_cell_and_half_cell_boundaries(precision, order):
    # exact integer and half-integer positions (shape tie-breaks, reading 14), moving
    # slowly so that they stay near them
    nx, ny = 32, 16
    rng = np.random.default_rng(170 + order)
    n = nx * ny
    xs = np.concatenate([np.arange(nx, dtype=float), np.arange(nx) + 0.5])
    ys = np.concatenate([np.arange(ny, dtype=float), np.arange(ny) + 0.5])
    x = rng.choice(xs, n)
    y = rng.choice(ys, n)
    sp = []
    for qm in (1.0, -1.0):
        sp.append({"qm": qm, "x": x.copy(), "y": y.copy(), "ux": rng.normal(0, 0.01, n),
                   "uy": rng.normal(0, 0.01, n), "uz": rng.normal(0, 0.01, n)})
    w = inputs.macro_weight(1, 1.0)
    F0 = inputs.random_fields(nx, ny, 0.05, seed=171)
    kw = {"tile_x": 16, "tile_y": 8} if precision == pic.PIC_MIXED32 else {}
    Fg, pg, _ = run_gpu(nx, ny, 1, sp, F0, 1, order, gamma0=1.0, cg_rtol=1e-13, precision=precision, **kw)
    Fo, po = oracle_run(nx, ny, w, sp, F0, 1, order, 1.0)
    tol = 1e-12 if precision == pic.PIC_FP64 else TOL32
    for c in range(9):
        check(Fg[c], Fo[c], tol, f"quantity {c}")


@pytest.mark.parametrize("nx,ny", [(4096, 8), (8, 2048), (1002, 24)])
@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_MIXED32])
def test_long_thin_grids_match_oracle(precision, nx, ny):
    ppc = 1
    w, sp = inputs.drifting_pair_plasma(nx, ny, ppc, 3.0, 0.3, seed=180, colocated=False)
    F0 = inputs.random_fields(nx, ny, 0.05, seed=181)
    Fg, pg, _ = run_gpu(nx, ny, ppc, sp, F0, 1, 2, gamma0=3.0, cg_rtol=1e-13, precision=precision)
    Fo, po = oracle_run(nx, ny, w, sp, F0, 1, 2, 1.0)
    tol = 1e-12 if precision == pic.PIC_FP64 else TOL32
    for c in range(9):
        check(Fg[c], Fo[c], tol, f"quantity {c}")
