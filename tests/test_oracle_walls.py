"""Pins of the oracle's conducting, reflecting walls at x = 0 and x = nx dx (the shock
configuration: the paper reflects the injected plasma at a wall, Sec. 4).

* the operator of Eq. (7) with walls is diagonalised by the discrete cosine transform
  (By, Bz: even images, Neumann) and the discrete sine transform (Bx: odd images,
  Dirichlet) in x and the FFT in y: the PCG must match that direct solve;
* standing vacuum modes of the conducting box follow the same exact amplification
  lambda(S) as plane waves (Eq. 10), with kx = pi m / (nx dx);
* a closed box conserves the field energy exactly at theta = 1/2 (no flux through a
  perfect conductor), which holds only if the discrete curls stay adjoint with walls;
* particles that cross a wall are reflected, and the folded deposit still satisfies
  the discrete continuity equation to round-off on every node off the wall."""
import math

import numpy as np
import pytest
from scipy import fft

import oracle
from closed_forms import amplification, relerr


def wall_solve(b3, nx, ny, theta, dt):
    """Direct solve of [1 - (theta dt)^2 Lap] x = b with the wall conditions: DST-I on the
    interior integer nodes 1..nx-1 for Bx, DCT-II on the half-integer nodes for By, Bz,
    FFT in y (dx = dy = 1)."""
    a = (theta * dt) ** 2
    ky = 2 * np.pi * np.fft.fftfreq(ny)
    lam_y = 4 * np.sin(ky / 2) ** 2
    out = np.zeros_like(b3)
    # Bx: odd images, zero on the wall nodes i = 0 (and i = nx, not stored)
    m = np.arange(1, nx)
    lam_x = 4 * np.sin(np.pi * m / (2 * nx)) ** 2
    bh = fft.dst(np.fft.fft(b3[0][:, 1:], axis=0), type=1, axis=1)
    xh = bh / (1 + a * (lam_y[:, None] + lam_x[None, :]))
    out[0][:, 1:] = np.real(np.fft.ifft(fft.idst(xh, type=1, axis=1), axis=0))
    # By, Bz: even images about the walls
    m = np.arange(nx)
    lam_x = 4 * np.sin(np.pi * m / (2 * nx)) ** 2
    for c in (1, 2):
        bh = fft.dct(np.fft.fft(b3[c], axis=0), type=2, axis=1)
        xh = bh / (1 + a * (lam_y[:, None] + lam_x[None, :]))
        out[c] = np.real(np.fft.ifft(fft.idct(xh, type=2, axis=1), axis=0))
    return out


@pytest.mark.parametrize("theta,cfl", [(0.5, 1.0), (0.501, 0.5), (0.75, 0.9)])
def test_pcg_with_walls_matches_cosine_sine_solve(theta, cfl):
    nx, ny = 24, 16
    g = oracle.grid(nx, ny, cfl, theta, 2, walls=True)
    rng = np.random.default_rng(3)
    b = rng.standard_normal((3, ny, nx))
    b[0][:, 0] = 0.0  # Bx on the wall is zero
    x, it, rr = oracle.pcg(g, b, rtol=1e-14, maxit=500)
    assert it > 0 and rr <= 1e-14
    assert relerr(x.reshape(3, ny, nx), wall_solve(b, nx, ny, theta, cfl)) < 1e-13


def test_wall_operator_is_symmetric():
    nx, ny = 16, 12
    g = oracle.grid(nx, ny, 0.9, 0.6, 1, walls=True)
    rng = np.random.default_rng(4)
    u, v = rng.standard_normal((2, 3, ny, nx))
    u[0][:, 0] = v[0][:, 0] = 0.0
    lhs = np.dot(u.ravel(), oracle.apply_A(g, v))
    rhs = np.dot(v.ravel(), oracle.apply_A(g, u))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def _box_te(nx, ny, mx, my):
    kx, ky = math.pi * mx / nx, 2 * math.pi * my / ny
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    F = np.zeros((6, ny, nx))
    F[5] = np.cos(kx * (ii + 0.5)) * np.cos(ky * (jj + 0.5))  # Bz, even about the walls
    return F, kx, ky


def _box_tm(nx, ny, mx, my):
    # B = curl(A_z z) with A_z = sin(kx x) cos(ky y) on the nodes: zero on the walls
    kx, ky = math.pi * mx / nx, 2 * math.pi * my / ny
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    A = np.sin(kx * ii) * np.cos(ky * jj)
    F = np.zeros((6, ny, nx))
    F[3] = np.roll(A, -1, axis=0) - A                                   # Bx = dA/dy
    Ae = np.concatenate([A, np.zeros((ny, 1))], axis=1)                 # A at i = nx is 0
    F[4] = -(Ae[:, 1:] - Ae[:, :-1])                                    # By = -dA/dx
    return F, kx, ky


@pytest.mark.parametrize("pol", ["TE", "TM"])
@pytest.mark.parametrize("theta,cfl", [(0.5, 1.0), (0.501, 0.7), (0.75, 1.0)])
def test_standing_modes_of_the_box_follow_the_dispersion_relation(pol, theta, cfl):
    nx, ny, nsteps = 24, 16, 10
    for mx, my in [(1, 0), (3, 1), (7, 5), (12, 8)]:
        F0, kx, ky = (_box_te if pol == "TE" else _box_tm)(nx, ny, mx, my)
        sim = oracle.OracleSim(nx, ny, cfl, theta, 1, [], cg_rtol=1e-15, fields=F0, walls=True)
        S = math.hypot(cfl * math.sin(kx / 2), cfl * math.sin(ky / 2))
        lam = amplification(theta, S)
        comp = [5] if pol == "TE" else [3, 4]
        for n in range(1, nsteps + 1):
            sim.step()
            for c in comp:
                np.testing.assert_allclose(sim.fields()[c], (lam ** n).real * F0[c], rtol=0, atol=2e-13)


def test_closed_box_conserves_energy_at_crank_nicolson():
    nx, ny = 20, 16
    rng = np.random.default_rng(5)
    F = rng.standard_normal((6, ny, nx))
    A = rng.standard_normal((ny, nx))
    A[:, 0] = 0.0
    Ae = np.concatenate([A, np.zeros((ny, 1))], axis=1)
    F[3] = np.roll(A, -1, axis=0) - A  # divergence-free B with Bx = 0 on the wall
    F[4] = -(Ae[:, 1:] - Ae[:, :-1])
    sim = oracle.OracleSim(nx, ny, 1.0, 0.5, 1, [], cg_rtol=1e-14, fields=F, walls=True)
    e0 = sum(sim.energies()[:2])
    for _ in range(30):
        sim.step()
    assert abs(sum(sim.energies()[:2]) - e0) < 1e-12 * e0
    assert np.all(sim.fields()[[1, 2, 3]][:, :, 0] == 0.0)  # Ey, Ez, Bx stay zero on the wall


def test_particle_reflects_at_the_walls():
    nx, ny = 16, 8
    g = oracle.grid(nx, ny, 1.0, 0.5, 2, walls=True)
    F = np.zeros(6 * nx * ny)
    x = np.array([0.3, nx - 0.2])
    y = np.array([4.0, 4.0])
    ux = np.array([-5.0, 5.0])
    uy = np.zeros(2)
    uz = np.array([0.3, -0.2])
    gam = np.sqrt(1 + ux ** 2 + uz ** 2)
    step = 1.0 * 5.0 / gam
    J, bad = oracle.push_deposit(g, F, 1.0, 1.0, x, y, ux, uy, uz)
    assert bad == 0
    np.testing.assert_allclose(x, [step[0] - 0.3, 2 * nx - (nx - 0.2 + step[1])], rtol=0, atol=1e-13)
    np.testing.assert_array_equal(ux, [5.0, -5.0])
    np.testing.assert_allclose(np.sqrt(1 + ux ** 2 + uz ** 2), gam, rtol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_folded_deposit_satisfies_continuity(p):
    nx, ny = 20, 12
    cfl = 0.95
    g = oracle.grid(nx, ny, cfl, 0.5, p, walls=True)
    rng = np.random.default_rng(30 + p)
    n = 3000
    F = rng.standard_normal((6, ny, nx)) * 0.3
    F[[1, 2, 3], :, 0] = 0.0
    x = np.concatenate([rng.uniform(0, 2.5, n // 2), rng.uniform(nx - 2.5, nx, n // 2)])
    y = rng.uniform(0, ny, n)
    ux = np.concatenate([-rng.uniform(1, 8, n // 2), rng.uniform(1, 8, n // 2)])
    uy, uz = rng.standard_normal((2, n)) * 2
    for qm in (1.0, -1.0):
        xs, ys = x.copy(), y.copy()
        rho0 = oracle.deposit_rho(g, 0.7 * qm, xs, ys)
        J, bad = oracle.push_deposit(g, F.ravel(), qm, 0.7 * qm, xs, ys, ux.copy(), uy.copy(), uz.copy())
        assert bad == 0
        assert xs.min() >= 0 and xs.max() < nx
        rho1 = oracle.deposit_rho(g, 0.7 * qm, xs, ys)
        # every node but the wall's, where the conductor takes up the surface charge
        resid = (rho1 - rho0 + cfl * oracle.div_J(g, J)).reshape(ny, nx)[:, 1:]
        assert np.abs(resid).max() < 1e-12



def test_gauss_law_holds_off_the_wall_with_reflecting_plasma():
    # a hot pair plasma bouncing between the walls: div E - 4 pi rho stays at its initial
    # value on every node off the wall (the wall node carries the conductor's surface
    # charge)
    nx, ny, ppc = 24, 12, 4
    rng = np.random.default_rng(9)
    species = []
    n = nx * ny * ppc
    for qm in (1.0, -1.0):
        species.append(oracle.Species(qm, 0.05, rng.uniform(0, nx, n), rng.uniform(0, ny, n),
                                      rng.standard_normal(n) * 3, rng.standard_normal(n),
                                      rng.standard_normal(n)))
    sim = oracle.OracleSim(nx, ny, 1.0, 0.5, 2, species, cg_rtol=1e-13, walls=True)

    def gauss():
        return (oracle.div_E(sim.g, sim.F) - 4 * math.pi * sim.rho()).reshape(ny, nx)[:, 1:]

    g0 = gauss()
    for _ in range(20):
        sim.step()
    assert sim.bad_moves == 0
    assert np.abs(gauss() - g0).max() < 1e-11
    for s in sim.species:
        assert s.x.min() >= 0 and s.x.max() < nx


# ---- the moving injector ---------------------------------------------------------------

def test_splitmix64_published_stream():
    # the splitmix64 stream seeded with 0 (Steele, Lea & Flood 2014): its first outputs
    z = np.array([0, 0x9E3779B97F4A7C15], dtype=np.uint64)
    assert [int(v) for v in oracle.splitmix64(z)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4]


def test_injector_counts_positions_and_momenta():
    nx, ny, cfl, x0, ppc, gamma0, u_th = 400, 16, 1.0, 4.0, 8, 10.0, 0.05
    w = (1 + math.sqrt(1 - 1 / gamma0 ** 2)) * cfl
    total, xs, mom = 0, [], []
    for n in range(300):
        new = oracle.inject_pairs(n, nx, ny, cfl, x0, ppc, gamma0, u_th, seed=7)
        xf = x0 + (n + 1) * cfl
        assert new is not None
        x, y, m = new
        total += x.size // ny
        assert total == math.floor(ppc * w * (n + 1))  # the beam's density over time
        assert np.all((x >= xf - w) & (x < xf)) and np.all(np.floor(y) == np.repeat(np.arange(ny), x.size // ny))
        xs.append((x - (xf - w)) / w)
        mom.append(m[0])
    assert oracle.inject_pairs(int(nx - x0), nx, ny, cfl, x0, ppc, gamma0, u_th, 7) is None
    u = np.concatenate(xs)
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1 / 12) < 0.003
    ux = np.concatenate([m[0] for m in mom])
    uy = np.concatenate([m[1] for m in mom])
    # back to the beam frame: u'x = gamma0 (ux + beta0 gamma) with ux toward -x
    beta0 = math.sqrt(1 - 1 / gamma0 ** 2)
    uz = np.concatenate([m[2] for m in mom])
    gam = np.sqrt(1 + ux ** 2 + uy ** 2 + uz ** 2)
    upx = -gamma0 * (ux + beta0 * gam)
    for comp in (upx, uy, uz):
        assert abs(comp.mean()) < 0.05 * u_th and abs(comp.std() / u_th - 1) < 0.05


def test_injected_beam_keeps_gauss_law():
    nx, ny, ppc = 48, 12, 4
    F = np.zeros((6, ny, nx))
    sim = oracle.OracleSim(nx, ny, 1.0, 0.5, 2, [oracle.Species(q, 0.05, [], [], [], [], []) for q in (1.0, -1.0)],
                           cg_rtol=1e-13, fields=F, walls=True,
                           injector=dict(x0=4.0, ppc=ppc, gamma0=5.0, u_th=0.1, seed=3))

    def gauss():
        return (oracle.div_E(sim.g, sim.F) - 4 * math.pi * sim.rho()).reshape(ny, nx)[:, 1:]

    g0 = gauss()
    for _ in range(25):
        sim.step()
    assert sim.species[0].n > 0 and sim.species[0].n == sim.species[1].n
    assert np.abs(gauss() - g0).max() < 1e-11
    assert sim.species[0].x.max() < nx
