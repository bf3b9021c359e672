"""Fourier diagnostics on the GPU (Sec. 3.1, Fig. 3): pic_spectrum against the oracle's
FFT amplitude (random fields on power-of-two, mixed-radix and prime-factor grids, the
2048 x 512 bench grid, and the charge density of a particle load), and the paper's
claim that numerical Cherenkov radiation grows on the resonance line of Eq. (17): a
run of the Sec. 3 configuration (Gamma = 100 flow, 10% thermal spread, order 2, theta
0.501, CFL 0.5, t = 230 dx/c) whose strongest B_z modes sit on the line."""
import math

import numpy as np
import pytest

import oracle
import paper_1412_2480_gb300 as pic
from paper_1412_2480_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nx,ny", [(64, 64), (72, 40), (22, 14), (8192, 8), (2048, 512)])
def test_spectrum_matches_oracle(nx, ny):
    F0 = inputs.random_fields(nx, ny, 1.0, seed=nx + ny)
    rng = np.random.default_rng(nx * ny)
    F0[5] += 0.1 * rng.standard_normal((ny, nx))  # broadband part
    prm = pic.pic_params_default(nx=nx, ny=ny)
    h = pic.pic_init(prm)
    try:
        pic.pic_set_fields(h, pic.PIC_BZ, np.ascontiguousarray(F0[5]).ravel())
        A = pic.pic_spectrum(h, pic.PIC_BZ, nx, ny)
    finally:
        pic.pic_free(h)
    ref = oracle.spectrum(F0[5])
    assert np.max(np.abs(A - ref)) <= 1e-12 * ref.max()


def test_spectrum_of_charge_density_matches_oracle():
    nx, ny, ppc = 48, 30, 3
    w, sp = inputs.drifting_pair_plasma(nx, ny, ppc, 3.0, 0.3, seed=12, colocated=False)
    prm = pic.pic_params_default(nx=nx, ny=ny, shape_order=2, gamma0=3.0, ppc=ppc)
    h = pic.pic_init(prm)
    try:
        for s, d in enumerate(sp):
            pic.pic_load_particles(h, s, d["x"], d["y"], d["ux"], d["uy"], d["uz"])
        A = pic.pic_spectrum(h, pic.PIC_RHO, nx, ny)
    finally:
        pic.pic_free(h)
    g = oracle.grid(nx, ny, 1.0, 0.5, 2)
    rho = np.zeros(nx * ny)
    for d in sp:
        oracle.deposit_rho(g, d["qm"] * w, d["x"], d["y"], rho)
    ref = oracle.spectrum(rho.reshape(ny, nx))
    assert np.max(np.abs(A - ref)) <= 1e-12 * ref.max()


def folded_wavenumbers(nx, ny):
    """k_x dx, k_y dy of every FFT index, folded to k_x >= 0 by the symmetry of a real
    field's spectrum (|F^(-k)| = |F^(k)|)."""
    p = np.arange(nx)
    q = np.arange(ny)
    kx = 2 * np.pi * np.where(p <= nx // 2, p, p - nx) / nx
    ky = 2 * np.pi * np.where(q <= ny // 2, q, q - ny) / ny
    KY, KX = np.meshgrid(ky, kx, indexing="ij")
    flip = KX < 0
    return np.where(flip, -KX, KX), np.where(flip, -KY, KY)


def test_cherenkov_modes_sit_on_the_resonance_line():
    nx = ny = 128
    cfl, gamma0, u_th, ppc, steps = 0.5, 100.0, 0.1, 100, 460  # t = 230 dx / c
    w, sp = inputs.drifting_pair_plasma(nx, ny, ppc, gamma0, u_th, seed=33)
    prm = pic.pic_params_default(nx=nx, ny=ny, cfl=cfl, theta=0.501, shape_order=2, gamma0=gamma0,
                                 ppc=ppc, precision=pic.PIC_MIXED32, cg_rtol=1e-8)
    h = pic.pic_init(prm)
    try:
        for s, d in enumerate(sp):
            pic.pic_load_particles(h, s, d["x"], d["y"], d["ux"], d["uy"], d["uz"])
        pic.pic_step(h, steps)
        m = pic.pic_moments(h)
        A = pic.pic_spectrum(h, pic.PIC_BZ, nx, ny)
    finally:
        pic.pic_free(h)
    beta = math.sqrt(1 - 1 / gamma0 ** 2)
    KX, KY = folded_wavenumbers(nx, ny)
    dk = 2 * np.pi / ny
    line = np.full(KX.shape, np.nan)
    for idx in np.ndindex(KX.shape):
        if KX[idx] > 0:
            v = pic.pic_resonance_ky(cfl, cfl, beta, KX[idx])
            if v is not None:
                line[idx] = v
    # band: within 3 grid wave numbers (3 x 2 pi / 128) of the line, about 6.5% of k-space
    on_line = np.abs(np.abs(KY) - line) <= 3 * dk  # NaN compares False
    power = A ** 2
    power[0, 0] = 0.0
    top = np.argsort(power.ravel())[::-1][:20]
    frac_top = float(np.mean(on_line.ravel()[top]))
    frac_power = float(power[on_line].sum() / power.sum())
    print(f"U_B/U_K = {m['U_B'] / m['U_K']:.3e}, top-20 on line {frac_top:.2f}, power on line {frac_power:.2f}, "
          f"band area {on_line.mean():.3f}")
    assert m["U_B"] > 1e-2 * m["U_K"]  # the instability has grown to saturation
    assert on_line.mean() < 0.08
    assert frac_top >= 0.75
    assert frac_power >= 0.5
