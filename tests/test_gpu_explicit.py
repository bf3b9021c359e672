"""Explicit FDTD field update (Eqs. 3-4, PIC_EXPLICIT), GPU against the oracle through
the C ABI: one step of a hot plasma in random fields (orders 1-3, periodic and walls;
FP64 to 1e-12, MIXED32 to 2e-5), a 100-step plasma run, vacuum modes on the recurrence
that Eq. (16) fixes, Gauss's law carried along, and the Courant-limit validation."""
import math

import numpy as np
import pytest

import paper_1412_2480_gb300 as pic
from paper_1412_2480_gb300 import inputs
from runners import check, check_rows, match_particles, rel, run_gpu, run_oracle, workload

pytestmark = pytest.mark.gpu
TOL32 = 2e-5


def hot(nx, ny, ppc, seed, walls):
    w, sp, F0 = workload(nx, ny, ppc, gamma0=3.0, u_th=0.3, seed=seed, field_amp=0.05,
                         colocated=False)
    if walls:
        F0 = F0.copy()
        F0[[1, 2, 3], :, 0] = 0.0
    return w, sp, F0


@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_MIXED32])
def test_explicit_step_matches_oracle(precision, order, walls):
    nx, ny, ppc, cfl = 40, 24, 3, 0.5
    w, sp, F0 = hot(nx, ny, ppc, 110 + order, walls)
    kw = {"tile_x": 16, "tile_y": 8} if precision == pic.PIC_MIXED32 else {}
    Fg, pg, mom = run_gpu(nx, ny, ppc, sp, F0, 1, order, cfl=cfl, gamma0=3.0, precision=precision,
                          flags=pic.PIC_EXPLICIT,
                          bc_x=pic.PIC_BC_WALLS if walls else pic.PIC_BC_PERIODIC, **kw)
    Fo, po, sim = run_oracle(nx, ny, w, sp, F0, 1, order, cfl=cfl, walls=walls, solver="explicit")
    tol = 1e-12 if precision == pic.PIC_FP64 else TOL32
    for c in range(9):  # E, B, J
        check(Fg[c], Fo[c], tol, f"quantity {c}")
    for s in range(2):
        d = match_particles(pg[s], po[s], [nx, ny, 3.0, 3.0, 3.0])
        assert d < (1e-12 if precision == pic.PIC_FP64 else 1e-5), d
    assert mom["cg_iters_last"] == 0


@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_MIXED32])
def test_explicit_plasma_run_matches_oracle(precision):
    nx, ny, ppc, steps, cfl = 32, 16, 4, 100, 0.5
    w, sp, F0 = workload(nx, ny, ppc, gamma0=20.0, u_th=1e-3, seed=120)
    kw = {"tile_x": 16, "tile_y": 8} if precision == pic.PIC_MIXED32 else {}
    Fg, pg, mom = run_gpu(nx, ny, ppc, sp, F0, steps, 2, cfl=cfl, precision=precision,
                          flags=pic.PIC_EXPLICIT, **kw)
    Fo, po, sim = run_oracle(nx, ny, w, sp, F0, steps, 2, cfl=cfl, solver="explicit")
    tol = 1e-9 if precision == pic.PIC_FP64 else 1e-3
    for c in range(6):
        assert rel(Fg[c], Fo[c]) < tol, f"field {c}: {rel(Fg[c], Fo[c]):.2e}"
    assert np.max(np.abs(Fg[3:6])) > 0  # the beam radiates


def test_explicit_vacuum_mode_recurrence():
    # f_{n+1} + f_{n-1} = 2 (1 - 2 (S_x^2 + S_y^2)) f_n for a single Fourier mode (Eq. 16)
    nx, ny, cfl, p, q = 64, 32, 0.6, 5, 3
    prm = pic.pic_params_default(nx=nx, ny=ny, cfl=cfl, flags=pic.PIC_EXPLICIT)
    h = pic.pic_init(prm)
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    bz = np.cos(2 * np.pi * (p * (i + 0.5) / nx + q * (j + 0.5) / ny))
    hist = []
    try:
        pic.pic_set_fields(h, pic.PIC_BZ, np.ascontiguousarray(bz).ravel())
        for _ in range(8):
            hist.append(pic.fields_numpy(h, pic.PIC_BZ, nx, ny))
            pic.pic_step(h, 1)
    finally:
        pic.pic_free(h)
    sx = cfl * math.sin(math.pi * p / nx)
    sy = cfl * math.sin(math.pi * q / ny)
    c = 1.0 - 2.0 * (sx * sx + sy * sy)
    for n in range(1, 7):
        assert np.max(np.abs(hist[n + 1] + hist[n - 1] - 2 * c * hist[n])) < 1e-12


@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_MIXED32])
def test_explicit_gauss_law_held(precision):
    nx, ny, ppc, gamma0 = 48, 32, 4, 3.0
    w, sp = inputs.drifting_pair_plasma(nx, ny, ppc, gamma0, 0.3, seed=131)
    prm = pic.pic_params_default(nx=nx, ny=ny, cfl=0.5, shape_order=2, gamma0=gamma0, ppc=ppc,
                                 precision=precision, flags=pic.PIC_EXPLICIT,
                                 tile_x=16 if precision == pic.PIC_MIXED32 else 0, tile_y=8)
    h = pic.pic_init(prm)
    try:
        for s, d in enumerate(sp):
            pic.pic_load_particles(h, s, d["x"], d["y"], d["ux"], d["uy"], d["uz"])
        pic.pic_step(h, 20)
        c1 = pic.pic_conservation(h)
    finally:
        pic.pic_free(h)
    s0 = 0.01 * gamma0
    assert c1["gauss_max"] <= (1e-12 if precision == pic.PIC_FP64 else 2e-4) * s0


def test_explicit_validation():
    with pytest.raises(pic.PicError):
        pic.pic_init(pic.pic_params_default(cfl=0.75, flags=pic.PIC_EXPLICIT))  # 2 cfl^2 > 1
    with pytest.raises(pic.PicError):
        pic.pic_init(pic.pic_params_default(cfl=0.5, flags=pic.PIC_EXPLICIT, precision=pic.PIC_MIXED32,
                                            warm_start=pic.PIC_WS_LEARNED))
    ps = [pic.pic_params_default(cfl=0.5, precision=pic.PIC_MIXED32, flags=pic.PIC_EXPLICIT),
          pic.pic_params_default(cfl=0.5, precision=pic.PIC_MIXED32)]
    with pytest.raises(pic.PicError):
        pic.pic_init_batch(ps)
    # at the limit: dx = dy, cfl = 1/sqrt(2) is accepted
    h = pic.pic_init(pic.pic_params_default(cfl=math.sqrt(0.5), flags=pic.PIC_EXPLICIT))
    pic.pic_free(h)
