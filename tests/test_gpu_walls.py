"""Conducting, reflecting walls in x (the shock configuration), GPU against the oracle
through the C ABI: one step of a hot plasma crossing both walls (FP64 to 1e-12, MIXED32
to 2e-5, orders 1-3), and a magnetised pair beam flowing into the wall at x = 0 over
many steps (the shock set-up of Sec. 4 mirrored), FP64 and MIXED32 against the oracle;
the MIXED32 shock run with overflowing bins reproduces itself bit for bit."""
import numpy as np
import pytest

import paper_1412_2480_gb300 as pic
from paper_1412_2480_gb300 import inputs
from runners import check, check_rows, match_particles, rel, run_gpu, run_oracle, workload

pytestmark = pytest.mark.gpu
TOL32 = 2e-5


def hot_near_walls(nx, ny, ppc, seed):
    """A hot plasma with random fields (zero on the wall column), particles near both
    walls moving into them."""
    w, sp, F0 = workload(nx, ny, ppc, gamma0=3.0, u_th=0.3, seed=seed, field_amp=0.05,
                         colocated=False)
    rng = np.random.default_rng(seed)
    for d in sp:
        n = d["x"].size
        left = rng.random(n) < 0.5
        d["x"] = np.where(left, rng.uniform(0, 2.0, n), rng.uniform(nx - 2.0, nx, n))
        d["ux"] = np.where(left, -np.abs(d["ux"]) - 1.0, np.abs(d["ux"]) + 1.0)
    F0 = F0.copy()
    F0[[1, 2, 3], :, 0] = 0.0
    return w, sp, F0


def sorted_particles(p):
    return p[:, np.lexsort(p[::-1])]


@pytest.mark.parametrize("order", [1, 2, 3])
def test_fp64_step_with_walls_matches_oracle(order):
    nx, ny, ppc = 40, 24, 3
    w, sp, F0 = hot_near_walls(nx, ny, ppc, 40 + order)
    Fg, pg, mom = run_gpu(nx, ny, ppc, sp, F0, 1, order, gamma0=3.0, cg_rtol=1e-13,
                          bc_x=pic.PIC_BC_WALLS)
    Fo, po, sim = run_oracle(nx, ny, w, sp, F0, 1, order, cg_rtol=1e-13, walls=True)
    for c in range(12):
        check(Fg[c], Fo[c], 1e-12, f"quantity {c}")
    for s in range(2):
        check_rows(pg[s], po[s], 1e-12, f"species {s}")
        assert pg[s][0].min() >= 0 and pg[s][0].max() < nx
    assert np.all(Fg[[1, 2, 3]][:, :, 0] == 0.0)  # Ey, Ez, Bx on the wall


@pytest.mark.parametrize("order", [1, 2, 3])
def test_mixed32_step_with_walls_matches_oracle(order):
    nx, ny, ppc = 40, 24, 3
    w, sp, F0 = hot_near_walls(nx, ny, ppc, 50 + order)
    Fg, pg, mom = run_gpu(nx, ny, ppc, sp, F0, 1, order, gamma0=3.0, cg_rtol=1e-13,
                          precision=pic.PIC_MIXED32, tile_x=16, tile_y=8, bc_x=pic.PIC_BC_WALLS)
    Fo, po, sim = run_oracle(nx, ny, w, sp, F0, 1, order, cg_rtol=1e-13, walls=True)
    for c in range(9):
        check(Fg[c], Fo[c], TOL32, f"quantity {c}")
    for s in range(2):
        g, o = sorted_particles(pg[s]), sorted_particles(po[s])
        assert np.max(np.abs(g[0] - o[0])) < TOL32 * nx
        check_rows(g[2:], o[2:], TOL32, f"species {s} momenta")
        assert g[0].min() >= 0 and g[0].max() < nx


@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_MIXED32])
def test_magnetised_beam_into_the_wall_matches_oracle(precision):
    # gamma0 = 10 pairs at sigma_B = 0.1 hit the wall at x = 0 and reflect; after 40
    # steps the reflected beam has built up the shock transition near the wall
    nx, ny, ppc, steps = 64, 16, 4, 40
    w, sp, F0 = inputs.shock_beam(nx, ny, ppc, 10.0, 1e-3, seed=5, sigma_b=0.1)
    kw = {} if precision == pic.PIC_FP64 else {"tile_x": 16, "tile_y": 8}
    Fg, pg, mom = run_gpu(nx, ny, ppc, sp, F0, steps, 2, gamma0=10.0, cg_rtol=1e-12,
                          precision=precision, bc_x=pic.PIC_BC_WALLS, **kw)
    Fo, po, sim = run_oracle(nx, ny, w, sp, F0, steps, 2, cg_rtol=1e-12, walls=True)
    tol = 1e-9 if precision == pic.PIC_FP64 else 1e-3
    for c in range(6):
        assert rel(Fg[c], Fo[c]) < tol, f"field {c}: {rel(Fg[c], Fo[c]):.2e}"
    # the beam reversed at the wall: some particles now move in +x
    assert np.any(pg[0][2] > 0) and np.any(po[0][2] > 0)
    # magnetic energy of the final fields (pic_moments reports the level the last step
    # started from, so compare the arrays themselves)
    ub_g, ub_o = np.sum(Fg[3:6] ** 2), sim.energies()[1] * 8 * np.pi
    assert abs(ub_g - ub_o) < tol * ub_o


def test_walls_validation_and_set_fields_zeroes_the_wall():
    prm = pic.pic_params_default(nx=16, ny=16, bc_x=pic.PIC_BC_WALLS)
    h = pic.pic_init(prm)
    try:
        data = np.ones(16 * 16)
        pic.pic_set_fields(h, pic.PIC_EY, data)
        out = pic.fields_numpy(h, pic.PIC_EY, 16, 16)
        assert np.all(out[:, 0] == 0.0) and np.all(out[:, 1:] == 1.0)
        with pytest.raises(pic.PicError) as e:
            pic.pic_load_particles(h, 0, np.array([16.5]), np.array([1.0]), np.zeros(1), np.zeros(1),
                                   np.zeros(1))
        assert e.value.code == pic.PIC_EINVAL
    finally:
        pic.pic_free(h)


def injector_setup(nx, ny, ppc, gamma0, seed):
    """The shock set-up with the moving injector: the magnetised beam behind the plane
    (x < x0), the fields of the beam everywhere (a static vacuum solution ahead)."""
    x0 = 12.0
    w, sp, F0 = inputs.shock_beam(nx, ny, ppc, gamma0, 1e-3, seed=seed, sigma_b=0.1)
    for d in sp:
        keep = d["x"] < x0
        for key in ("x", "y", "ux", "uy", "uz"):
            d[key] = np.ascontiguousarray(d[key][keep])
    inj = dict(x0=x0, ppc=ppc, gamma0=gamma0, u_th=1e-3, seed=11)
    return w, sp, F0, inj


def run_oracle_injected(nx, ny, w, sp, F0, steps, order, inj):
    import oracle
    species = [oracle.Species(d["qm"], w, d["x"], d["y"], d["ux"], d["uy"], d["uz"]) for d in sp]
    sim = oracle.OracleSim(nx, ny, 1.0, 0.5, order, species, cg_rtol=1e-12, fields=F0, walls=True,
                           injector=inj)
    sim.step(steps)
    return sim


@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_MIXED32])
def test_moving_injector_matches_oracle(precision):
    nx, ny, ppc, steps, gamma0 = 64, 16, 4, 30, 10.0
    w, sp, F0, inj = injector_setup(nx, ny, ppc, gamma0, seed=9)
    kw = {} if precision == pic.PIC_FP64 else {"tile_x": 16, "tile_y": 8}
    Fg, pg, mom = run_gpu(nx, ny, ppc, sp, F0, steps, 2, gamma0=gamma0, cg_rtol=1e-12,
                          precision=precision, bc_x=pic.PIC_BC_WALLS, inject_x0=inj["x0"],
                          u_th=inj["u_th"], seed=inj["seed"], **kw)
    sim = run_oracle_injected(nx, ny, w, sp, F0, steps, 2, inj)
    n_o = sim.species[0].n
    assert n_o > sum(d["x"].size for d in sp[:1])  # the injector added pairs
    assert mom["n_particles"] == (n_o, n_o)
    tol = 1e-9 if precision == pic.PIC_FP64 else 1e-3
    Fo = sim.fields()
    for c in range(6):
        assert rel(Fg[c], Fo[c]) < tol, f"field {c}: {rel(Fg[c], Fo[c]):.2e}"
    for s in range(2):
        o = np.stack([sim.species[s].x, sim.species[s].y, sim.species[s].ux, sim.species[s].uy,
                      sim.species[s].uz])
        d = match_particles(pg[s], o, [nx, ny, gamma0, gamma0, gamma0])
        assert d < (1e-10 if precision == pic.PIC_FP64 else 1e-4), d


def test_mixed32_shock_with_overflow_is_bit_reproducible():
    # The beam piles up against the wall and bins with little slack overflow. Which
    # particles find no room depends on warp scheduling; a parked particle is pushed
    # from global memory with the rounding of its tile's current window, so the run
    # alone and two copies of it in one batch (other tile order, other overflow) agree
    # bit for bit.
    nx, ny, ppc, steps, gamma0 = 64, 16, 6, 24, 10.0
    w, sp, F0, inj = injector_setup(nx, ny, ppc, gamma0, seed=5)
    prm = dict(nx=nx, ny=ny, cfl=1.0, theta=0.5, shape_order=2, gamma0=gamma0, ppc=ppc,
               precision=pic.PIC_MIXED32, cg_rtol=1e-12, tile_x=8, tile_y=8, bin_slack=1.05,
               bc_x=pic.PIC_BC_WALLS, inject_x0=inj["x0"], u_th=inj["u_th"], seed=inj["seed"])

    def load(h):
        for c in range(6):
            pic.pic_set_fields(h, c, np.ascontiguousarray(F0[c]).ravel())
        for s, d in enumerate(sp):
            pic.pic_load_particles(h, s, d["x"], d["y"], d["ux"], d["uy"], d["uz"])

    def state(h):
        F = np.stack([pic.fields_numpy(h, c, nx, ny) for c in range(12)])
        return F, [sorted_particles(pic.pic_particles(h, s)) for s in range(2)], pic.pic_moments(h)

    h = pic.pic_init(pic.pic_params_default(**prm))
    try:
        load(h)
        pic.pic_step(h, steps)
        runs = [state(h)]
    finally:
        pic.pic_free(h)
    h = pic.pic_init_batch([pic.pic_params_default(**prm) for _ in range(2)])
    try:
        for k in range(2):
            pic.pic_select(h, k)
            load(h)
        pic.pic_step(h, steps)
        for k in range(2):
            pic.pic_select(h, k)
            runs.append(state(h))
    finally:
        pic.pic_free(h)
    assert sum(m["overflow_moves"] for _, _, m in runs) > 0
    Fa, Pa, ma = runs[0]
    assert ma["n_particles"][0] > sum(d["x"].size for d in sp[:1])  # the injector added pairs
    for Fb, Pb, mb in runs[1:]:
        assert mb["n_particles"] == ma["n_particles"]
        for q in range(12):
            assert np.array_equal(Fa[q], Fb[q]), f"quantity {q}"
        for s in range(2):
            assert np.array_equal(Pa[s], Pb[s]), f"species {s}"
