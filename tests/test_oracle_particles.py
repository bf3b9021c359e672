"""Pins of the oracle's particle half: shapes, gather, Boris push, Esirkepov deposit.

Each test ties the oracle to something other than itself: scipy's B-splines, the
B-spline moment identities, the exact rotation of the Boris scheme in a uniform B,
the discrete continuity equation with an independently computed charge density, the
closed-form current moments, and the tau-integral definition of the density
decomposition."""
import math

import numpy as np
import pytest

import oracle
from closed_forms import bspline, div_nodes

ORDERS = (1, 2, 3)


@pytest.mark.parametrize("p", ORDERS)
def test_shape_is_centred_bspline(p):
    d = np.linspace(-2.6, 2.6, 1041)
    ref = bspline(p)(d)
    got = oracle.shape(p, d)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("p", ORDERS)
def test_shape_moments(p):
    # partition of unity and linear precision: sum_k W(x-k) = 1, sum_k k W(x-k) = x
    rng = np.random.default_rng(1)
    for x in rng.uniform(-3, 3, 50):
        k = np.arange(math.floor(x) - 3, math.floor(x) + 4)
        w = oracle.shape(p, x - k)
        assert abs(w.sum() - 1) < 1e-14
        assert abs((k * w).sum() - x) < 1e-13


OFFS = [(0.5, 0.0), (0.0, 0.5), (0.0, 0.0), (0.0, 0.5), (0.5, 0.0), (0.5, 0.5)]


@pytest.mark.parametrize("p", ORDERS)
def test_gather_uniform_and_linear_fields(p):
    nx, ny = 32, 24
    g = oracle.grid(nx, ny, 1.0, 0.5, p)
    rng = np.random.default_rng(2)
    # uniform field: reproduced exactly anywhere (partition of unity)
    F = np.zeros((6, ny, nx))
    vals = rng.standard_normal(6)
    for c in range(6):
        F[c] = vals[c]
    x = rng.uniform(0, nx, 200)
    y = rng.uniform(0, ny, 200)
    got = oracle.gather(g, F, x, y)
    np.testing.assert_allclose(got, np.repeat(vals[:, None], 200, 1), rtol=1e-14, atol=1e-14)
    # linear field in the lattice coordinates: reproduced exactly away from the wrap
    a, bx, by = rng.standard_normal(3)
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    for c, (ox, oy) in enumerate(OFFS):
        F[c] = a + bx * (ii + ox) + by * (jj + oy) + c
    x = rng.uniform(5, nx - 5, 200)
    y = rng.uniform(5, ny - 5, 200)
    got = oracle.gather(g, F, x, y)
    for c in range(6):
        np.testing.assert_allclose(got[c], a + bx * x + by * y + c, rtol=1e-13, atol=1e-12)


def test_gather_staggered_offsets_distinct():
    # A single nonzero node value must be felt by a particle at that component's
    # own staggered position, with weight W(0)^2.
    nx = ny = 16
    for p in ORDERS:
        g = oracle.grid(nx, ny, 1.0, 0.5, p)
        w0 = oracle.shape(p, np.array([0.0]))[0]
        for c, (ox, oy) in enumerate(OFFS):
            F = np.zeros((6, ny, nx))
            F[c, 7, 5] = 1.0
            got = oracle.gather(g, F, np.array([5 + ox]), np.array([7 + oy]))
            assert abs(got[c, 0] - w0 * w0) < 1e-15
            assert np.all(np.delete(got[:, 0], c) == 0)


def rodrigues(k, a, v):
    k = k / np.linalg.norm(k)
    return v * math.cos(a) + np.cross(k, v) * math.sin(a) + k * np.dot(k, v) * (1 - math.cos(a))


@pytest.mark.parametrize("qm", [1.0, -1.0])
def test_boris_exact_gyration(qm):
    # E = 0, uniform B: the Boris rotation turns u by exactly 2 atan(|t|) per step,
    # |t| = (q/m)(dt/2)|B|/gamma, in the sense of u x B for q > 0.
    rng = np.random.default_rng(3)
    B0 = np.array([0.3, -0.5, 0.8])
    dt = 0.7
    u0 = rng.standard_normal(3) * 5
    u = u0[None, :].copy()
    gam = math.sqrt(1 + u0 @ u0)
    phi = 2 * math.atan(0.5 * dt * np.linalg.norm(B0) / gam)
    for n in range(1, 41):
        u = oracle.boris(qm, dt, np.zeros((1, 3)), B0[None, :], u)
        ref = rodrigues(B0, -math.copysign(1, qm) * n * phi, u0)
        np.testing.assert_allclose(u[0], ref, rtol=0, atol=1e-12 * np.linalg.norm(u0))
    assert abs(np.linalg.norm(u[0]) - np.linalg.norm(u0)) < 1e-13 * np.linalg.norm(u0)


def test_boris_pure_electric_kick():
    rng = np.random.default_rng(4)
    E = rng.standard_normal((10, 3))
    u0 = rng.standard_normal((10, 3))
    for qm in (1.0, -1.0):
        u = oracle.boris(qm, 0.37, E, np.zeros((10, 3)), u0)
        np.testing.assert_allclose(u, u0 + qm * 0.37 * E, rtol=0, atol=1e-15)


def _boris_by_rotation(qm, dt, E, B, u):
    """One Boris step written as what its t/s construction amounts to: a half electric
    kick, an exact rotation of u- about B by 2 atan(|h||B|/gamma-) (Rodrigues' formula,
    sense of u x B for q > 0), where gamma- = sqrt(1 + |u-|^2) is taken AFTER the first
    kick, then the second half kick. Independent of the oracle's cross products."""
    h = 0.5 * qm * dt
    um = u + h * E
    gm = math.sqrt(1.0 + um @ um)
    bn = np.linalg.norm(B)
    if bn == 0.0:
        return um + h * E
    phi = 2.0 * math.atan(abs(h) * bn / gm)
    return rodrigues(B, -math.copysign(1.0, qm) * phi, um) + h * E


@pytest.mark.parametrize("qm", [1.0, -1.0])
def test_boris_parallel_e_and_b_closed_form(qm):
    # E parallel to B: the kicks act along B only, so u_par gains exactly (q/m) dt |E|
    # per step, while u_perp keeps its length and turns by 2 atan(|h||B|/gamma-) with
    # gamma- = sqrt(1 + |u^{n-1/2} + h E|^2). A gamma from u^{n-1/2} (before the first
    # kick) gives a different angle at every step and fails this.
    rng = np.random.default_rng(6)
    bhat = np.array([0.36, -0.48, 0.8])
    B = 1.7 * bhat
    E = 0.9 * bhat
    dt = 0.6
    h = 0.5 * qm * dt
    u = rng.standard_normal(3) * 3
    upar = u @ bhat
    uperp = u - upar * bhat
    for n in range(1, 31):
        gm = math.sqrt(1.0 + (upar + h * 0.9) ** 2 + uperp @ uperp)
        uperp = rodrigues(bhat, -math.copysign(1.0, qm) * 2.0 * math.atan(abs(h) * 1.7 / gm), uperp)
        upar = upar + 2.0 * h * 0.9
        u = oracle.boris(qm, dt, E[None, :], B[None, :], u[None, :])[0]
        assert abs(u @ bhat - upar) < 1e-12 * max(1.0, abs(upar))
        np.testing.assert_allclose(u - (u @ bhat) * bhat, uperp, rtol=0, atol=1e-12 * np.linalg.norm(uperp))


@pytest.mark.parametrize("qm", [1.0, -1.0])
def test_boris_crossed_e_and_b_against_rotation_form(qm):
    # E perpendicular (and oblique) to B, relativistic momenta: every step equals the
    # kick - exact rotation - kick sequence written independently above. Applying the
    # second kick before the rotation, or one full kick, or gamma of u^{n-1/2}, all
    # fail here because the kick does not commute with the rotation.
    rng = np.random.default_rng(7)
    dt = 0.45
    for trial in range(20):
        B = rng.standard_normal(3) * 2
        E = np.cross(B, rng.standard_normal(3)) if trial % 2 == 0 else rng.standard_normal(3)
        u = rng.standard_normal(3) * 4
        for _ in range(25):
            ref = _boris_by_rotation(qm, dt, E, B, u)
            u = oracle.boris(qm, dt, E[None, :], B[None, :], u[None, :])[0]
            np.testing.assert_allclose(u, ref, rtol=0, atol=2e-13 * max(1.0, np.linalg.norm(ref)))


def test_boris_exb_drift():
    # Uniform E perpendicular to B with |E| << |B|: averaged over whole gyrations the
    # velocity u/gamma approaches the drift E x B / |B|^2 for either charge sign
    # (non-relativistic limit of the exact motion).
    B = np.array([0.0, 0.0, 1.0])
    E = np.array([0.0, 2e-3, 0.0])
    dt = 0.05
    vd = np.cross(E, B) / (B @ B)
    for qm in (1.0, -1.0):
        u = np.array([[0.0, 0.0, 0.0]])
        nper = int(round(2 * math.pi / dt))  # one gyration per 2 pi (gamma = 1 + O(1e-6))
        vs = []
        for _ in range(40 * nper):
            u = oracle.boris(qm, dt, E[None, :], B[None, :], u)
            g = math.sqrt(1.0 + (u[0] @ u[0]))
            vs.append(u[0] / g)
        vbar = np.mean(vs, axis=0)
        np.testing.assert_allclose(vbar, vd, rtol=0, atol=2e-2 * np.linalg.norm(vd))


def _rho_scipy(p, nx, ny, q, x, y):
    W = bspline(p)
    rho = np.zeros((ny, nx))
    for xi, yi in zip(np.atleast_1d(x), np.atleast_1d(y)):
        i = np.arange(math.floor(xi) - 3, math.floor(xi) + 4)
        j = np.arange(math.floor(yi) - 3, math.floor(yi) + 4)
        wx, wy = W(xi - i), W(yi - j)
        np.add.at(rho, (np.mod(j, ny)[:, None], np.mod(i, nx)[None, :]), q * np.outer(wy, wx))
    return rho


def _quadrature_current(p, nx, ny, q, dt, x0, y0, x1, y1, vz):
    """Density decomposition by its defining tau integrals (3-point Gauss, exact here):
    Wx = int_0^1 DSx (S0y + tau DSy), Wy likewise, Wz = int_0^1 (S0x + tau DSx)(S0y + tau DSy);
    Jx = -q dx/dt/(dx dy) cumsum_x Wx, Jy likewise along y, Jz = q vz Wz/(dx dy)."""
    W = bspline(p)
    i = np.arange(math.floor(min(x0, x1)) - 3, math.floor(min(x0, x1)) + 6)
    j = np.arange(math.floor(min(y0, y1)) - 3, math.floor(min(y0, y1)) + 6)
    S0x, S1x, S0y, S1y = W(x0 - i), W(x1 - i), W(y0 - j), W(y1 - j)
    DSx, DSy = S1x - S0x, S1y - S0y
    tau, wq = np.polynomial.legendre.leggauss(3)
    tau, wq = 0.5 * (tau + 1), 0.5 * wq
    Wx = sum(w * np.outer(S0y + t * DSy, DSx) for t, w in zip(tau, wq))
    Wy = sum(w * np.outer(DSy, S0x + t * DSx) for t, w in zip(tau, wq))
    Wz = sum(w * np.outer(S0y + t * DSy, S0x + t * DSx) for t, w in zip(tau, wq))
    J = np.zeros((3, ny, nx))
    idx = (np.mod(j, ny)[:, None], np.mod(i, nx)[None, :])
    np.add.at(J[0], idx, -q / dt * np.cumsum(Wx, axis=1))
    np.add.at(J[1], idx, -q / dt * np.cumsum(Wy, axis=0))
    np.add.at(J[2], idx, q * vz * Wz)
    return J


@pytest.mark.parametrize("p", ORDERS)
def test_esirkepov_single_particle(p):
    nx, ny, dt = 16, 16, 0.9
    g = oracle.grid(nx, ny, dt, 0.5, p)
    rng = np.random.default_rng(10 + p)
    for _ in range(40):
        x0, y0 = rng.uniform(0, nx), rng.uniform(0, ny)
        dxm, dym = rng.uniform(-0.999, 0.999, 2)
        x1, y1 = x0 + dxm, y0 + dym
        vz = rng.standard_normal()
        q = rng.choice([-1.0, 1.0]) * rng.uniform(0.1, 2)
        J = oracle.deposit_move(g, q, x0, y0, x1, y1, vz).reshape(3, ny, nx)
        # (a) discrete continuity with an independently computed rho (scipy shapes)
        rho0 = _rho_scipy(p, nx, ny, q, x0, y0)
        rho1 = _rho_scipy(p, nx, ny, q, x1 % nx, y1 % ny)
        resid = rho1 - rho0 + dt * div_nodes(J[:2])
        assert np.abs(resid).max() < 1e-14 * max(1, abs(q) / dt)
        # (b) closed-form current moments: sum J dx dy = q v
        np.testing.assert_allclose(J[0].sum(), q * dxm / dt, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(J[1].sum(), q * dym / dt, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(J[2].sum(), q * vz, rtol=1e-12, atol=1e-14)
        # (c) tau-integral definition of the decomposition
        Jq = _quadrature_current(p, nx, ny, q, dt, x0, y0, x1, y1, vz)
        np.testing.assert_allclose(J, Jq, rtol=0, atol=1e-13 * max(1, abs(q) / dt))


@pytest.mark.parametrize("p", ORDERS)
def test_push_deposit_continuity_many_particles(p):
    # Random fields and momenta; rho from the oracle's own charge assignment (pinned to
    # scipy above); the deposit must satisfy rho^{n+1} - rho^n + dt div J = 0.
    nx, ny = 24, 20
    cfl = 0.95
    g = oracle.grid(nx, ny, cfl, 0.5, p)
    rng = np.random.default_rng(20 + p)
    n = 3000
    F = rng.standard_normal(6 * nx * ny) * 0.3
    x, y = rng.uniform(0, nx, n), rng.uniform(0, ny, n)
    ux, uy, uz = rng.standard_normal((3, n)) * 3
    for qm in (1.0, -1.0):
        xs, ys = x.copy(), y.copy()
        rho0 = oracle.deposit_rho(g, 0.7 * qm, xs, ys)
        J, bad = oracle.push_deposit(g, F, qm, 0.7 * qm, xs, ys, ux.copy(), uy.copy(), uz.copy())
        assert bad == 0
        assert xs.min() >= 0 and xs.max() < nx and ys.min() >= 0 and ys.max() < ny
        rho1 = oracle.deposit_rho(g, 0.7 * qm, xs, ys)
        resid = rho1 - rho0 + cfl * oracle.div_J(g, J)
        assert np.abs(resid).max() < 1e-12


def test_colocated_pairs_with_equal_momenta_give_zero_current():
    nx = ny = 16
    g = oracle.grid(nx, ny, 1.0, 0.5, 2)
    rng = np.random.default_rng(5)
    n = 500
    x, y = rng.uniform(0, nx, n), rng.uniform(0, ny, n)
    u = rng.standard_normal((3, n))
    J = np.zeros(3 * nx * ny)
    F = np.zeros(6 * nx * ny)
    for qm in (1.0, -1.0):
        oracle.push_deposit(g, F, qm, qm * 0.3, x.copy(), y.copy(), u[0].copy(), u[1].copy(),
                            u[2].copy(), J)
    assert np.abs(J).max() < 1e-15
