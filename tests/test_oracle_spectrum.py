"""Pins of the oracle's Fourier diagnostics (Sec. 3.1, Fig. 3): the amplitude spectrum
against the brute-force DFT sum, Parseval's identity and single modes; the resonance
line of Eq. (17) against the dispersion relation Eq. (15) it is derived from; and the
C ABI's host-side resonance function against the oracle's (no GPU needed)."""
import math

import numpy as np
import pytest

import oracle


def brute_dft_amplitude(F):
    ny, nx = F.shape
    out = np.zeros((ny, nx))
    l = np.arange(nx)
    m = np.arange(ny)
    for q in range(ny):
        for p in range(nx):
            ph = np.exp(-2j * np.pi * (np.outer(m * q / ny, np.ones(nx)) + np.outer(np.ones(ny), l * p / nx)))
            out[q, p] = abs(np.sum(F * ph)) / F.size
    return out


def test_spectrum_equals_the_brute_force_sum():
    rng = np.random.default_rng(1)
    F = rng.standard_normal((6, 10))
    assert np.max(np.abs(oracle.spectrum(F) - brute_dft_amplitude(F))) < 1e-13


def test_spectrum_parseval_and_single_mode():
    rng = np.random.default_rng(2)
    F = rng.standard_normal((24, 40))
    A = oracle.spectrum(F)
    # Parseval: sum |F^|^2 = N sum |F|^2, with A = |F^| / N
    assert abs(np.sum((A * F.size) ** 2) - F.size * np.sum(F * F)) < 1e-9 * F.size * np.sum(F * F)
    # cos(2 pi (3 l / nx + 5 m / ny)) puts 1/2 at (p, q) = (3, 5) and (nx - 3, ny - 5)
    ny, nx = 24, 40
    m, l = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    A = oracle.spectrum(np.cos(2 * np.pi * (3 * l / nx + 5 * m / ny)))
    assert abs(A[5, 3] - 0.5) < 1e-14 and abs(A[ny - 5, nx - 3] - 0.5) < 1e-14
    A[5, 3] = A[ny - 5, nx - 3] = 0.0
    assert A.max() < 1e-14


@pytest.mark.parametrize("cfl", [0.5, 0.7, 1.0])
@pytest.mark.parametrize("beta", [0.9999, 0.99])
def test_resonance_line_lies_on_both_dispersion_surfaces(cfl, beta):
    # on the line, omega = V k_x satisfies tan^2(omega dt / 2) = S_x^2 + S_y^2 (Eq. 15)
    found = 0
    for kx in np.linspace(0.05, math.pi, 60):
        ky = oracle.resonance_ky(cfl, cfl, beta, kx)
        if ky is None:
            continue
        found += 1
        w_dt = beta * kx * cfl
        sx, sy = cfl * math.sin(kx / 2), cfl * math.sin(ky / 2)
        assert abs(math.tan(w_dt / 2) ** 2 - sx * sx - sy * sy) < 1e-12 * (1 + math.tan(w_dt / 2) ** 2)
        assert 0.0 <= ky <= math.pi
    assert found > 0


def test_resonance_line_absent_where_the_flow_is_slower_than_the_waves():
    # at long wavelength the scheme's waves move at nearly c > V: no crossing; at
    # beta -> 0 no crossing anywhere
    assert oracle.resonance_ky(0.5, 0.5, 0.9999, 0.01) is None
    assert all(oracle.resonance_ky(0.5, 0.5, 0.1, k) is None for k in np.linspace(0.1, math.pi, 20))


def test_capi_resonance_matches_oracle():
    # the library's host-side Eq. (17) against the oracle's, on a sweep
    import paper_1412_2480_gb300 as pic
    from paper_1412_2480_gb300 import build
    build.build()
    for cfl in (0.4, 0.5, 0.8, 1.0):
        for beta in (0.9, 0.9999):
            for kx in np.linspace(0.02, math.pi, 50):
                a = pic.pic_resonance_ky(cfl, cfl, beta, kx)
                b = oracle.resonance_ky(cfl, cfl, beta, kx)
                assert (a is None) == (b is None), (cfl, beta, kx)
                if a is not None:
                    assert abs(a - b) <= 1e-14 * max(1.0, b)
