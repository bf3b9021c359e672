"""Pins of the oracle's field half: RHS of Eq. (7), its operator, the PCG solve and the
update from Eqs. (5)-(6).

* the operator of Eq. (7) against its Fourier symbol and the PCG against a direct FFT
  solve (library routine, special case of the periodic grid);
* vacuum plane waves against the exact root of the paper's dispersion relation Eq. (10),
  and at theta = 1/2 against Eq. (15) itself, for both polarisations;
* the update must satisfy the paper's time discretisation Eqs. (5)-(6), checked with
  independent numpy.roll Yee operators;
* energy: exactly conserved in vacuum at theta = 1/2 (Crank-Nicolson), decaying for
  theta > 1/2 (the damping claim below Eq. (12));
* div B stays at round-off."""
import math

import numpy as np
import pytest

import oracle
from closed_forms import (S_xy, amplification, curl_of_B_lattice, curl_of_E_lattice,
                          eq10_residual, eq11_real, eq12_imag, k2_symbol, relerr,
                          spectral_solve)


def test_amplification_solves_eq10_and_eq15():
    for theta in (0.5, 0.501, 0.6, 0.75, 1.0):
        for S in (0.05, 0.3, 0.7, 1.0, 1.4):
            lam = amplification(theta, S)
            assert abs(eq10_residual(theta, lam, S / math.sqrt(2), S / math.sqrt(2))) < 1e-13
            assert abs(lam) <= 1 + 1e-15
            if theta > 0.5:
                assert abs(lam) < 1  # damping for theta > 1/2 (text below Eq. (12))
    # theta = 1/2: tan^2(omega dt / 2) = Sx^2 + Sy^2 (Eq. (15)), |lambda| = 1
    for S in (0.1, 0.5, 1.0, 1.3):
        lam = amplification(0.5, S)
        assert abs(abs(lam) - 1) < 1e-15
        assert abs(math.tan(np.angle(lam) / 2) ** 2 - S * S) < 1e-13
        # the paper's Eqs. (11)-(12) are exact at theta = 1/2
        assert abs(eq11_real(0.5, S) - np.angle(lam)) < 1e-13
        assert abs(eq12_imag(0.5, S)) < 1e-15
    # Reading of Eqs. (11)-(12): they are 2 atan(Re tan(omega dt/2)) and
    # 2 atan(Im tan(omega dt/2)) of the exact root, not Re/Im of omega dt itself. Near
    # theta = 1/2 (the paper's optimum 0.501, Sec. 3.3) Eq. (11) matches arg(lambda) to
    # 1e-5 and Eq. (12) exceeds the true damping -ln|lambda| by the factor 1 + S^2.
    for theta in (0.501, 0.6, 1.0):
        for S in (0.2, 0.6, 1.0):
            lam = amplification(theta, S)
            t = np.tan(-1j * np.log(lam) / 2)
            assert abs(eq11_real(theta, S) - 2 * math.atan(t.real)) < 1e-12
            assert abs(eq12_imag(theta, S) - 2 * math.atan(t.imag)) < 1e-12
            if theta == 0.501:
                assert abs(eq11_real(theta, S) - np.angle(lam)) < 1e-5
                damp = -math.log(abs(lam))
                assert damp > 0 and eq12_imag(theta, S) > 0
                assert abs(eq12_imag(theta, S) / (1 + S * S) - damp) < 1e-3 * damp


def test_operator_fourier_symbol():
    nx, ny, theta, dt = 24, 16, 0.6, 0.8
    g = oracle.grid(nx, ny, dt, theta, 1)
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    for mx, my in [(0, 0), (1, 0), (3, 2), (12, 8), (5, 7)]:
        kx, ky = 2 * math.pi * mx / nx, 2 * math.pi * my / ny
        v = np.cos(kx * ii + ky * jj)
        x = np.stack([v, 2 * v, -v])
        eig = 1 + (theta * dt) ** 2 * (4 * math.sin(kx / 2) ** 2 + 4 * math.sin(ky / 2) ** 2)
        np.testing.assert_allclose(oracle.apply_A(g, x).reshape(3, ny, nx), eig * x,
                                   rtol=0, atol=1e-13)


@pytest.mark.parametrize("theta,cfl", [(0.5, 1.0), (0.501, 0.5), (0.75, 0.9), (1.0, 1.0)])
def test_pcg_matches_spectral_solve(theta, cfl):
    nx, ny = 40, 24
    g = oracle.grid(nx, ny, cfl, theta, 2)
    rng = np.random.default_rng(7)
    b = rng.standard_normal((3, ny, nx))
    x, it, rr = oracle.pcg(g, b, rtol=1e-14, maxit=500)
    assert it > 0 and rr <= 1e-14
    ref = spectral_solve(b, nx, ny, theta, cfl)
    assert relerr(x.reshape(3, ny, nx), ref) < 5e-14
    # warm start from the answer converges immediately; zero rhs gives zero
    x2, it2, _ = oracle.pcg(g, b, x0=ref, rtol=1e-12)
    assert it2 == 0
    x3, it3, rr3 = oracle.pcg(g, np.zeros((3, ny, nx)), x0=np.ones(3 * nx * ny))
    assert it3 == 0 and rr3 == 0 and np.all(x3 == 0)


def _te_mode(nx, ny, mx, my):
    kx, ky = 2 * math.pi * mx / nx, 2 * math.pi * my / ny
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    F = np.zeros((6, ny, nx))
    F[5] = np.cos(kx * (ii + 0.5) + ky * (jj + 0.5))  # Bz at (i+1/2, j+1/2)
    return F, kx, ky


def _tm_mode(nx, ny, mx, my):
    # B = curl(A_z z), A_z = cos(k.x) at nodes: discretely divergence-free by construction
    kx, ky = 2 * math.pi * mx / nx, 2 * math.pi * my / ny
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    A = np.cos(kx * ii + ky * jj)
    F = np.zeros((6, ny, nx))
    F[3] = np.roll(A, -1, axis=0) - A  # Bx at (i, j+1/2) = dA/dy
    F[4] = -(np.roll(A, -1, axis=1) - A)  # By at (i+1/2, j) = -dA/dx
    return F, kx, ky


@pytest.mark.parametrize("pol", ["TE", "TM"])
@pytest.mark.parametrize("theta,cfl", [(0.5, 1.0), (0.5, 0.5), (0.501, 1.0), (0.75, 0.7),
                                       (1.0, 1.0)])
def test_vacuum_mode_follows_dispersion_relation(pol, theta, cfl):
    nx, ny, nsteps = 32, 16, 12
    for mx, my in [(1, 0), (3, 1), (7, 5), (16, 0), (11, 8)]:
        F0, kx, ky = (_te_mode if pol == "TE" else _tm_mode)(nx, ny, mx, my)
        sim = oracle.OracleSim(nx, ny, cfl, theta, 1, [], cg_rtol=1e-15, fields=F0)
        Sx, Sy = S_xy(cfl, cfl, kx, ky)
        lam = amplification(theta, math.hypot(Sx, Sy))
        comp = [5] if pol == "TE" else [3, 4]
        for n in range(1, nsteps + 1):
            sim.step()
            amp = (lam**n).real
            for c in comp:
                np.testing.assert_allclose(sim.fields()[c], amp * F0[c], rtol=0, atol=2e-13)
        if theta == 0.5:
            # Eq. (15): the phase advance per step is 2 atan(S)
            assert abs(np.angle(lam) - 2 * math.atan(math.hypot(Sx, Sy))) < 1e-14


def test_time_discretisation_eqs_5_and_6_hold():
    # random divergence-free B (curl of a random A_z plus a random Bz), random E and J;
    # after one field solve+update, Eq. (5) and Eq. (6) hold with independent operators.
    nx, ny, theta, cfl = 20, 28, 0.55, 0.9
    rng = np.random.default_rng(8)
    A = rng.standard_normal((ny, nx))
    F = np.zeros((6, ny, nx))
    F[:3] = rng.standard_normal((3, ny, nx))
    F[3] = np.roll(A, -1, axis=0) - A
    F[4] = -(np.roll(A, -1, axis=1) - A)
    F[5] = rng.standard_normal((ny, nx))
    J = rng.standard_normal((3, ny, nx))
    g = oracle.grid(nx, ny, cfl, theta, 2)
    b = oracle.rhs(g, F, J)
    dB, it, rr = oracle.pcg(g, b, rtol=1e-15, maxit=500)
    F1 = oracle.field_update(g, F, dB, J).reshape(6, ny, nx)
    dt = cfl
    E0, B0, E1, B1 = F[:3], F[3:], F1[:3], F1[3:]
    lhs5 = (B1 - B0) / dt
    rhs5 = -curl_of_E_lattice(theta * E1 + (1 - theta) * E0)
    assert relerr(lhs5, rhs5) < 1e-13
    lhs6 = (E1 - E0) / dt
    rhs6 = curl_of_B_lattice(theta * B1 + (1 - theta) * B0) - 4 * math.pi * J
    assert relerr(lhs6, rhs6) < 1e-13
    assert np.abs(oracle.div_B(g, F1)).max() < 1e-12


def _random_vacuum_fields(nx, ny, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((ny, nx))
    F = np.zeros((6, ny, nx))
    F[3] = np.roll(A, -1, axis=0) - A
    F[4] = -(np.roll(A, -1, axis=1) - A)
    F[5] = rng.standard_normal((ny, nx))
    F[:3] = rng.standard_normal((3, ny, nx))
    return F


def test_vacuum_energy_conserved_at_crank_nicolson_and_damped_above():
    nx, ny = 24, 24
    F0 = _random_vacuum_fields(nx, ny, 9)
    sim = oracle.OracleSim(nx, ny, 1.0, 0.5, 2, [], cg_rtol=1e-15, fields=F0)
    e0 = sum(sim.energies()[:2])
    for _ in range(20):
        sim.step()
    assert abs(sum(sim.energies()[:2]) - e0) < 1e-12 * e0
    sim = oracle.OracleSim(nx, ny, 1.0, 0.6, 2, [], cg_rtol=1e-15, fields=F0)
    prev = e0
    for _ in range(10):
        sim.step()
        cur = sum(sim.energies()[:2])
        assert cur < prev
        prev = cur


def test_k2_symbol_pins_laplacian_sign():
    # the spectral symbol used above is positive (minus the Laplacian), so the
    # eigenvalues of Eq. (7)'s operator are >= 1: the matrix is SPD.
    s = k2_symbol(8, 8)
    assert s.min() == 0 and s.max() > 7.9
