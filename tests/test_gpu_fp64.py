"""FP64 CUDA path vs the oracle, element by element, through the C ABI.

Tolerance: single-step fields, currents and momenta within 1e-12 relative (norm-wise;
FP64 atomics sum in a different order than the oracle, so results agree to rounding).
Sizes span several field blocks with a ragged tail (72 x 40 = 2880 cells = 11.25 blocks
of 256) and several particle blocks with a ragged tail."""
import math

import numpy as np
import pytest

import paper_1412_2480_gb300 as pic
from closed_forms import amplification
from runners import check, check_rows, periodic_pos_err, rel, run_gpu, run_oracle, workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("steps", [1, 4])
def test_fp64_step_matches_oracle(order, steps):
    nx, ny, ppc = 72, 40, 3
    w, sp, F0 = workload(nx, ny, ppc, gamma0=5.0, u_th=0.2, seed=order, field_amp=0.05,
                         colocated=False)
    Fg, pg, mom = run_gpu(nx, ny, ppc, sp, F0, steps, order, gamma0=5.0, cg_rtol=1e-13)
    Fo, po, sim = run_oracle(nx, ny, w, sp, F0, steps, order, cg_rtol=1e-13)
    assert mom["macro_weight"] == pytest.approx(w, rel=1e-15)
    assert mom["step"] == steps
    for c in range(6):
        check(Fg[c], Fo[c], 1e-12, f"field {c}")
    for c in range(6, 9):
        check(Fg[c], Fo[c], 1e-12, f"current {c - 6}")
    for c in range(9, 12):
        check(Fg[c], Fo[c], 1e-12, f"dB {c - 9}")
    for s in range(2):
        assert periodic_pos_err(pg[s][0], po[s][0], nx) < 1e-12
        assert periodic_pos_err(pg[s][1], po[s][1], ny) < 1e-12
        check_rows(pg[s][2:], po[s][2:], 1e-12, f"species {s} momenta")
    assert mom["cg_iters_last"] == sim.last_cg_iters


def test_fp64_config1_shape_ten_steps():
    # 64 x 64, CFL 1, theta 1/2, order 1, gamma0 = 20, 1e-3 spread, 8 ppc per species
    nx = ny = 64
    w, sp, F0 = workload(nx, ny, 8, gamma0=20.0, u_th=1e-3, seed=1)
    Fg, pg, mom = run_gpu(nx, ny, 8, sp, F0, 10, 1, gamma0=20.0)
    Fo, po, sim = run_oracle(nx, ny, w, sp, F0, 10, 1)
    scale = np.linalg.norm(Fo[:6])
    assert scale > 0
    assert np.linalg.norm(Fg[:6] - Fo[:6]) / scale < 1e-10
    for s in range(2):
        assert rel(pg[s][2:], po[s][2:]) < 1e-12


@pytest.mark.parametrize("pol", ["TE", "TM"])
def test_fp64_vacuum_mode_closed_form(pol):
    # Pins the GPU field solve directly to Eq. (10)'s root, no oracle involved.
    nx, ny, theta, cfl = 48, 32, 0.75, 0.9
    mx, my = 5, 3
    kx, ky = 2 * math.pi * mx / nx, 2 * math.pi * my / ny
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    F0 = np.zeros((6, ny, nx))
    if pol == "TE":
        F0[5] = np.cos(kx * (ii + 0.5) + ky * (jj + 0.5))
        comps = [5]
    else:
        A = np.cos(kx * ii + ky * jj)
        F0[3] = np.roll(A, -1, axis=0) - A
        F0[4] = -(np.roll(A, -1, axis=1) - A)
        comps = [3, 4]
    S = cfl * math.hypot(math.sin(kx / 2), math.sin(ky / 2))
    lam = amplification(theta, S)
    for n in (1, 7):
        Fg, _, _ = run_gpu(nx, ny, 1, [], F0, n, 2, cfl=cfl, theta=theta, cg_rtol=1e-14,
                           want_particles=False)
        for c in comps:
            np.testing.assert_allclose(Fg[c], (lam**n).real * F0[c], rtol=0, atol=1e-12)


def test_fp64_warm_start_and_direct_launch():
    nx, ny, ppc = 40, 24, 2
    w, sp, F0 = workload(nx, ny, ppc, gamma0=3.0, u_th=0.3, seed=5, field_amp=0.1, colocated=False)
    Fo, po, _ = run_oracle(nx, ny, w, sp, F0, 3, 2, cg_rtol=1e-13, warm_start="prev")
    Fg, pg, mom = run_gpu(nx, ny, ppc, sp, F0, 3, 2, gamma0=3.0, cg_rtol=1e-13,
                          warm_start=pic.PIC_WS_PREV)
    Fd, pd, _ = run_gpu(nx, ny, ppc, sp, F0, 3, 2, gamma0=3.0, cg_rtol=1e-13,
                        warm_start=pic.PIC_WS_PREV, flags=pic.PIC_NO_GRAPH)
    assert rel(Fg[:9], Fo[:9]) < 1e-12
    assert rel(Fd[:9], Fg[:9]) < 1e-13
    assert rel(pd[0][2:], pg[0][2:]) < 1e-14


def test_fp64_error_paths():
    nx = ny = 32
    w, sp, F0 = workload(nx, ny, 2, gamma0=3.0, u_th=0.3, seed=6, field_amp=0.1, colocated=False)
    h = pic.pic_init(pic.pic_params_default(nx=nx, ny=ny, ppc=2, gamma0=3.0, cg_max_iter=1,
                                            cg_rtol=1e-14))
    try:
        for c in range(6):
            pic.pic_set_fields(h, c, np.ascontiguousarray(F0[c]).ravel())
        d = sp[0]
        pic.pic_load_particles(h, 0, d["x"], d["y"], d["ux"], d["uy"], d["uz"])
        with pytest.raises(pic.PicError) as e:
            pic.pic_step(h, 5)
        assert e.value.code == pic.PIC_ECG_NOCONV
        m = pic.pic_moments(h)
        assert m["step"] == 1  # the failing step completed, the rest were skipped
        bad = d["x"].copy()
        bad[3] = np.nan
        with pytest.raises(pic.PicError) as e:
            pic.pic_load_particles(h, 1, bad, d["y"], d["ux"], d["uy"], d["uz"])
        assert e.value.code == pic.PIC_EINVAL
        with pytest.raises(pic.PicError):
            pic.pic_set_fields(h, 9, np.zeros(nx * ny))
    finally:
        pic.pic_free(h)


def test_fp64_empty_species_and_zero_fields():
    # no particles, zero fields: b = 0, the solve returns dB = 0 and nothing moves
    nx, ny = 16, 16
    Fg, _, mom = run_gpu(nx, ny, 1, [], np.zeros((6, ny, nx)), 3, 1, want_particles=False)
    assert np.all(Fg == 0)
    assert mom["cg_iters_last"] == 0 and mom["step"] == 3
