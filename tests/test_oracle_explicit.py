"""Pins of the oracle's explicit FDTD update, Eqs. (3)-(4): single vacuum modes follow
the explicit dispersion relation Eq. (16) exactly; the Courant limit that Eq. (16)
implies (|sin| <= 1) separates bounded from growing runs; the first step from rest
reproduces the current coupling of Eq. (4) and the curl of Eq. (3) in closed form; and
Gauss's law is carried along by a plasma run with the charge-conserving deposit."""
import math

import numpy as np
import pytest

import oracle
from paper_1412_2480_gb300 import inputs


def mode_fields(nx, ny, p, q, comp):
    """A cosine of wave numbers (2 pi p / nx, 2 pi q / ny) on component comp's lattice."""
    F = np.zeros((6, ny, nx))
    off = {0: (0.5, 0.0), 1: (0.0, 0.5), 2: (0.0, 0.0), 3: (0.0, 0.5), 4: (0.5, 0.0), 5: (0.5, 0.5)}[comp]
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    F[comp] = np.cos(2 * np.pi * (p * (i + off[0]) / nx + q * (j + off[1]) / ny))
    return F


@pytest.mark.parametrize("cfl", [0.3, 0.5, 0.7])
@pytest.mark.parametrize("p,q,comp", [(1, 0, 5), (3, 2, 5), (2, 5, 2), (7, 3, 2), (4, 4, 5)])
def test_vacuum_mode_follows_eq16(cfl, p, q, comp):
    # On one Fourier mode the update is a 2x2 map with eigenvalues exp(-+ i w dt), so any
    # component obeys f_{n+1} + f_{n-1} = 2 cos(w dt) f_n, and Eq. (16) gives
    # cos(w dt) = 1 - 2 sin^2(w dt / 2) = 1 - 2 (S_x^2 + S_y^2).
    nx, ny = 16, 12
    g = oracle.grid(nx, ny, cfl, 0.5, 1)
    F = mode_fields(nx, ny, p, q, comp).ravel()
    J = np.zeros(3 * nx * ny)
    hist = [F.copy()]
    for _ in range(12):
        F = oracle.explicit_update(g, F, J)
        hist.append(F.copy())
    sx = cfl * math.sin(math.pi * p / nx)
    sy = cfl * math.sin(math.pi * q / ny)
    c = 1.0 - 2.0 * (sx * sx + sy * sy)
    for n in range(1, 12):
        resid = hist[n + 1] + hist[n - 1] - 2.0 * c * hist[n]
        assert np.max(np.abs(resid)) < 1e-12


def test_courant_limit():
    # Eq. (16) has real w for every mode only while S_x^2 + S_y^2 <= 1, i.e. 2 cfl^2 <= 1
    # at dx = dy: below it random fields stay bounded, above it the (pi, pi) mode grows
    nx = ny = 16
    F0 = inputs.random_fields(nx, ny, 1.0, seed=3).ravel()
    F0 += 1e-3 * np.random.default_rng(3).standard_normal(F0.size)
    J = np.zeros(3 * nx * ny)
    growth = {}
    for cfl in (0.70, 0.72):
        g = oracle.grid(nx, ny, cfl, 0.5, 1)
        F = F0.copy()
        for _ in range(400):
            F = oracle.explicit_update(g, F, J)
        growth[cfl] = np.linalg.norm(F) / np.linalg.norm(F0)
    assert growth[0.70] < 10.0
    assert growth[0.72] > 1e6


def test_first_step_from_rest_closed_form():
    # E = B = 0 and a current J: B^{1/2} = 0, E^1 = -4 pi dt J exactly (Eq. 4), and
    # B^1 = -(dt/2) curl E^1 = 2 pi dt^2 curl J, here for J_z = cos(a i + b j) on the
    # integer lattice: (curl J)_x at (i, j+1/2) = [cos(a i + b (j+1)) - cos(a i + b j)] / dy
    # and (curl J)_y at (i+1/2, j) = -[cos(a (i+1) + b j) - cos(a i + b j)] / dx
    nx, ny, dt = 16, 12, 0.5
    g = oracle.grid(nx, ny, dt, 0.5, 1)
    a, b = 2 * np.pi * 3 / nx, 2 * np.pi * 2 / ny
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    J = np.zeros((3, ny, nx))
    J[2] = np.cos(a * i + b * j)
    F = oracle.explicit_update(g, np.zeros(6 * nx * ny), J.ravel()).reshape(6, ny, nx)
    assert np.max(np.abs(F[2] + 4 * np.pi * dt * J[2])) < 1e-14
    assert np.max(np.abs(F[:2])) == 0.0
    cjx = np.cos(a * i + b * (j + 1)) - np.cos(a * i + b * j)
    cjy = -(np.cos(a * (i + 1) + b * j) - np.cos(a * i + b * j))
    assert np.max(np.abs(F[3] - 2 * np.pi * dt * dt * cjx)) < 1e-13
    assert np.max(np.abs(F[4] - 2 * np.pi * dt * dt * cjy)) < 1e-13
    assert np.max(np.abs(F[5])) == 0.0


@pytest.mark.parametrize("walls", [False, True])
def test_gauss_law_carried_by_a_plasma_run(walls):
    nx, ny, ppc = 24, 16, 3
    w, sp = inputs.drifting_pair_plasma(nx, ny, ppc, 3.0, 0.3, seed=21, colocated=False)
    species = [oracle.Species(d["qm"], w, d["x"], d["y"], d["ux"], d["uy"], d["uz"]) for d in sp]
    sim = oracle.OracleSim(nx, ny, 0.5, 0.5, 2, species, walls=walls, solver="explicit")

    def gauss():
        r = (oracle.div_E(sim.g, sim.F) - 4 * np.pi * sim.rho()).reshape(ny, nx)
        return r[:, 1:] if walls else r

    r0 = gauss()
    sim.step(30)
    assert np.max(np.abs(gauss() - r0)) < 1e-12 * max(1.0, np.max(np.abs(sim.rho())))
    assert np.max(np.abs(sim.F)) > 0.0
