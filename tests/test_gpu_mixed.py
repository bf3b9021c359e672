"""MIXED32 CUDA path (int cell + FP32 offset, FP32 gather/push/deposit, FP64 field solve)
vs the FP64 oracle on the same seeded inputs, through the C ABI.

Tolerance (2e-5, FP32 mode): applied relative to the scale of the terms each result is
summed from, which is the bound FP32 arithmetic can promise. For momenta and fields
that is their own norm. For the current of a co-located pair plasma, where positron
and electron currents cancel to ~1e-6 of either, it is the norm of one species' current.

Particles come back in tile order, so they are matched to the oracle's by nearest
neighbour in (x, y, ux, uy, uz); positions are compared modulo the box."""
import math

import numpy as np
import pytest

import oracle
import paper_1412_2480_gb300 as pic
from runners import check, check_rows, rel, run_gpu, run_oracle, workload

pytestmark = pytest.mark.gpu
TOL32 = 2e-5


def match(pg, po, nx, ny):
    """Index into pg for each oracle particle (nearest in position-momentum space)."""
    from scipy.spatial import cKDTree
    su = max(np.abs(po[2:]).max(), 1e-30)
    # unwrap-safe: use sin/cos embedding of the periodic coordinates
    def emb(p):
        return np.stack([np.cos(2 * np.pi * p[0] / nx) * nx, np.sin(2 * np.pi * p[0] / nx) * nx,
                         np.cos(2 * np.pi * p[1] / ny) * ny, np.sin(2 * np.pi * p[1] / ny) * ny,
                         p[2] / su, p[3] / su, p[4] / su], axis=1)
    tree = cKDTree(emb(pg))
    d, idx = tree.query(emb(po))
    assert len(np.unique(idx)) == po.shape[1], "particle matching is not one-to-one"
    return idx


def pos_err(a, b, L):
    d = np.abs(a - b)
    return float(np.max(np.minimum(d, L - d)))


@pytest.mark.parametrize("order", [1, 2, 3])
def test_mixed_step_matches_oracle(order):
    nx, ny, ppc = 72, 40, 3  # 3 x 3 tiles of 32 x 16, ragged in both directions
    w, sp, F0 = workload(nx, ny, ppc, gamma0=5.0, u_th=0.2, seed=10 + order, field_amp=0.05,
                         colocated=False)
    Fg, pg, mom = run_gpu(nx, ny, ppc, sp, F0, 1, order, gamma0=5.0, cg_rtol=1e-13,
                          precision=pic.PIC_MIXED32, tile_x=32, tile_y=16)
    Fo, po, sim = run_oracle(nx, ny, w, sp, F0, 1, order, cg_rtol=1e-13)
    assert mom["n_particles"] == (nx * ny * ppc, nx * ny * ppc)
    for c in range(6):
        check(Fg[c], Fo[c], TOL32, f"field {c}")
    for c in range(6, 9):
        check(Fg[c], Fo[c], TOL32, f"current {c - 6}")
    for c in range(9, 12):
        check(Fg[c], Fo[c], TOL32, f"dB {c - 9}")
    for s in range(2):
        idx = match(pg[s], po[s], nx, ny)
        g = pg[s][:, idx]
        assert pos_err(g[0], po[s][0], nx) < TOL32
        assert pos_err(g[1], po[s][1], ny) < TOL32
        check_rows(g[2:], po[s][2:], TOL32, f"species {s} momenta")


def test_mixed_colocated_pair_plasma_currents():
    # the production workload shape (co-located pairs, gamma0 = 20, 1e-3 spread)
    nx = ny = 64
    ppc = 8
    w, sp, F0 = workload(nx, ny, ppc, gamma0=20.0, u_th=1e-3, seed=1)
    Fg, pg, mom = run_gpu(nx, ny, ppc, sp, F0, 1, 1, gamma0=20.0, precision=pic.PIC_MIXED32,
                          tile_x=16, tile_y=8)
    Fo, po, sim = run_oracle(nx, ny, w, sp, F0, 1, 1)
    Jp, _, _ = run_oracle(nx, ny, w, sp[:1], F0, 1, 1)  # one species' current: the scale
    scale = np.linalg.norm(Jp[6:9])
    assert np.linalg.norm(Fg[6:9] - Fo[6:9]) / scale < TOL32
    e_scale = 4 * math.pi * sim.g.dt * scale
    assert np.linalg.norm(Fg[:3] - Fo[:3]) / e_scale < TOL32
    # element-wise against the largest current of one species: the deposit sums shape
    # differences DS = S1 - S0 of O(1) weights, which FP32 offsets resolve to ~6e-8
    # absolute whatever the move, so every component's error scales with the current of
    # a full-cell move (here Jx), not with a component's own size (Jy of this beam, whose
    # transverse moves are ~5e-5 cells, is ~1e-6 of Jx)
    jmax = np.abs(Jp[6:9]).max()
    for c in range(3):
        check(Fg[6 + c], Fo[6 + c], TOL32, f"current {c}", scale=jmax)
        check(Fg[c], Fo[c], TOL32, f"field {c}", scale=4 * math.pi * sim.g.dt * jmax)
    for s in range(2):
        idx = match(pg[s], po[s], nx, ny)
        check_rows(pg[s][2:, idx], po[s][2:], TOL32, f"species {s} momenta")


def test_mixed_many_steps_conserve_charge_and_particles():
    # 20 steps: every particle crosses tiles (drift ~1 cell/step with 8-cell tiles);
    # Gauss's law residual div E - 4 pi rho stays constant (Esirkepov) to FP32 level.
    nx, ny, ppc = 48, 24, 4
    w, sp, F0 = workload(nx, ny, ppc, gamma0=3.0, u_th=0.3, seed=3, colocated=False)
    prm = pic.pic_params_default(nx=nx, ny=ny, ppc=ppc, gamma0=3.0, shape_order=2,
                                 precision=pic.PIC_MIXED32, tile_x=8, tile_y=8)
    g = oracle.grid(nx, ny, 1.0, 0.5, 2)
    h = pic.pic_init(prm)
    try:
        for s in range(2):
            d = sp[s]
            pic.pic_load_particles(h, s, d["x"], d["y"], d["ux"], d["uy"], d["uz"])

        def gauss():
            F = np.stack([pic.fields_numpy(h, c, nx, ny) for c in range(6)])
            rho = np.zeros(nx * ny)
            for s in range(2):
                p = pic.pic_particles(h, s)
                oracle.deposit_rho(g, (1 if s == 0 else -1) * w, p[0], p[1], rho)
            return oracle.div_E(g, F) - 4 * math.pi * rho, rho

        g0, rho0 = gauss()
        for _ in range(4):
            pic.pic_step(h, 5)
            m = pic.pic_moments(h)
            assert m["n_particles"] == (nx * ny * ppc, nx * ny * ppc)
            assert m["cfl_violations"] == 0
            gk, rho = gauss()
            scale = 4 * math.pi * np.abs(rho).max() + 4 * math.pi * w
            assert np.abs(gk - g0).max() < 1e-5 * scale
        assert m["step"] == 20
    finally:
        pic.pic_free(h)


def test_mixed_bin_overflow_path_matches_oracle():
    # Counter-streaming halves pile up in the middle tiles, exceeding bins sized with
    # little slack: particles go through the overflow path and are re-sorted after the
    # call; results still match the oracle.
    nx, ny, ppc = 64, 16, 6
    w, sp, F0 = workload(nx, ny, ppc, gamma0=2.0, u_th=0.01, seed=4, colocated=False)
    for d in sp:
        left = d["x"] < nx / 2
        d["ux"] = np.where(left, 6.0, -6.0) + d["ux"] * 0
    Fg, pg, mom = run_gpu(nx, ny, ppc, sp, F0, 6, 1, gamma0=2.0, cg_rtol=1e-13,
                          precision=pic.PIC_MIXED32, tile_x=8, tile_y=8, bin_slack=1.05)
    Fo, po, sim = run_oracle(nx, ny, w, sp, F0, 6, 1, cg_rtol=1e-13)
    assert mom["overflow_moves"] > 0 and mom["rebins"] >= 1
    assert rel(Fg[6:9], Fo[6:9]) < 1e-4
    for s in range(2):
        idx = match(pg[s], po[s], nx, ny)
        assert pos_err(pg[s][0, idx], po[s][0], nx) < 1e-4


def test_mixed_empty_and_single_species():
    nx, ny = 16, 16
    Fg, pg, mom = run_gpu(nx, ny, 1, [], np.zeros((6, ny, nx)), 2, 2,
                          precision=pic.PIC_MIXED32, want_particles=False)
    assert np.all(Fg == 0) and mom["n_particles"] == (0, 0)
    w, sp, F0 = workload(nx, ny, 2, gamma0=3.0, u_th=0.3, seed=8, field_amp=0.05, colocated=False)
    Fg, pg, mom = run_gpu(nx, ny, 2, sp[:1], F0, 2, 2, gamma0=3.0, precision=pic.PIC_MIXED32,
                          cg_rtol=1e-13)
    Fo, po, _ = run_oracle(nx, ny, w, sp[:1], F0, 2, 2, cg_rtol=1e-13)
    assert rel(Fg[:9], Fo[:9]) < TOL32
    for c in range(9):
        check(Fg[c], Fo[c], TOL32, f"quantity {c}")


@pytest.mark.parametrize("theta,cfl,flags,rtol", [(0.5, 1.0, 0, 1e-13), (0.75, 0.9, 0, 1e-13),
                                                  (1.0, 1.0, 0, 1e-13), (0.5, 1.0, pic.PIC_CG_INNER, 1e-13),
                                                  (0.5, 1.0, 0, 1e-14)])
def test_mixed_precision_field_solve_meets_fp64_tolerance(theta, cfl, flags, rtol):
    # The MIXED32 solve refines FP32 inner solves (Chebyshev tiles; the inner CG with
    # PIC_CG_INNER, and for rtol 1e-14, below what the tiles' pair residual resolves)
    # against an FP64-class residual, so the vacuum mode must still follow the exact root
    # of Eq. (10) to FP64 accuracy.
    import math
    from closed_forms import amplification
    nx, ny, mx, my = 48, 32, 5, 3
    kx, ky = 2 * math.pi * mx / nx, 2 * math.pi * my / ny
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    F0 = np.zeros((6, ny, nx))
    F0[5] = np.cos(kx * (ii + 0.5) + ky * (jj + 0.5))
    lam = amplification(theta, cfl * math.hypot(math.sin(kx / 2), math.sin(ky / 2)))
    for n in (1, 6):
        Fg, _, mom = run_gpu(nx, ny, 1, [], F0, n, 2, cfl=cfl, theta=theta, cg_rtol=rtol,
                             precision=pic.PIC_MIXED32, want_particles=False, flags=flags)
        np.testing.assert_allclose(Fg[5], (lam**n).real * F0[5], rtol=0, atol=1e-12)
        assert 0 < mom["cg_rel_resid"] <= rtol


@pytest.mark.parametrize("order", [1, 3])
def test_cooperative_solve_agrees_with_graph_loop_solve(order):
    # the one-kernel cooperative PCG (with PIC_CG_INNER) and the WHILE-node PCG run the
    # same mixed-precision iteration; their reductions are partitioned differently, so
    # they agree to the solver tolerance rather than bit for bit
    nx, ny, ppc = 96, 64, 3
    w, sp, F0 = workload(nx, ny, ppc, gamma0=5.0, u_th=0.2, seed=30 + order, field_amp=0.05,
                         colocated=False)
    Fc, pc, mc = run_gpu(nx, ny, ppc, sp, F0, 3, order, gamma0=5.0, cg_rtol=1e-12,
                         precision=pic.PIC_MIXED32, flags=pic.PIC_CG_INNER)
    Fl, pl, ml = run_gpu(nx, ny, ppc, sp, F0, 3, order, gamma0=5.0, cg_rtol=1e-12,
                         precision=pic.PIC_MIXED32, flags=pic.PIC_NO_COOP)
    for c in range(12):
        assert rel(Fc[c], Fl[c]) < 1e-9, c
    assert mc["cg_rel_resid"] <= 1e-12 and ml["cg_rel_resid"] <= 1e-12
    assert abs(mc["cg_iters_total"] - ml["cg_iters_total"]) <= 3


@pytest.mark.parametrize("nx,ny,walls", [(96, 64, False), (200, 72, False), (96, 40, True), (16, 12, False)])
def test_chebyshev_inner_solve_agrees_with_cg(nx, ny, walls):
    # the Chebyshev tiles and the inner CG solve the same FP64-refined system to the same
    # FP64 tolerance, on grids with ragged tiles (200 x 72), conducting walls, and a grid
    # smaller than one tile and its halo (16 x 12, the window wraps around it)
    ppc, order = 3, 2
    w, sp, F0 = workload(nx, ny, ppc, gamma0=5.0, u_th=0.2, seed=7 + nx, field_amp=0.05, colocated=False)
    kw = dict(gamma0=5.0, cg_rtol=1e-12, precision=pic.PIC_MIXED32)
    if walls:
        kw["bc_x"] = pic.PIC_BC_WALLS
        for d in sp:
            d["x"] = np.clip(d["x"], 1e-3, nx - 1e-3)
        F0 = F0.copy()
        F0[1][:, 0] = F0[2][:, 0] = F0[3][:, 0] = 0.0  # Ey, Ez, Bx vanish on the wall nodes
    Fc, pc, mc = run_gpu(nx, ny, ppc, sp, F0, 3, order, **kw)
    Fg, pg, mg = run_gpu(nx, ny, ppc, sp, F0, 3, order, flags=pic.PIC_CG_INNER, **kw)
    for c in range(12):
        assert rel(Fc[c], Fg[c]) < 1e-9, c
    assert mc["cg_rel_resid"] <= 1e-12 and mg["cg_rel_resid"] <= 1e-12
    assert mc["cg_refinements"] >= 1 and mc["cg_iters_total"] > 0


def test_chebyshev_inner_solve_is_independent_of_the_batch():
    # a simulation's Chebyshev tiles read only its own cells: alone or in a batch with an
    # unlike neighbour it gives the same fields bit for bit
    nx, ny, ppc = 64, 64, 3
    w, sp, F0 = workload(nx, ny, ppc, gamma0=5.0, u_th=0.2, seed=5, field_amp=0.05, colocated=False)
    prm = [pic.pic_params_default(nx=nx, ny=ny, shape_order=2, gamma0=5.0, ppc=ppc, cg_rtol=1e-12,
                                  precision=pic.PIC_MIXED32),
           pic.pic_params_default(nx=96, ny=32, shape_order=1, gamma0=5.0, ppc=ppc, cg_rtol=1e-12,
                                  precision=pic.PIC_MIXED32, cfl=0.7)]
    out = []
    for batch in (False, True):
        h = pic.pic_init_batch(prm) if batch else pic.pic_init(prm[0])
        try:
            pic.pic_select(h, 0) if batch else None
            for c in range(6):
                pic.pic_set_fields(h, c, np.ascontiguousarray(F0[c]).ravel())
            for s, d in enumerate(sp):
                pic.pic_load_particles(h, s, d["x"], d["y"], d["ux"], d["uy"], d["uz"])
            pic.pic_step(h, 3)
            pic.pic_select(h, 0) if batch else None
            out.append(np.stack([pic.fields_numpy(h, c, nx, ny) for c in range(12)]))
        finally:
            pic.pic_free(h)
    assert np.array_equal(out[0], out[1])


def test_batch_rejects_unlike_handle_flags():
    prm = [pic.pic_params_default(nx=32, ny=32, precision=pic.PIC_MIXED32),
           pic.pic_params_default(nx=32, ny=32, precision=pic.PIC_MIXED32, flags=pic.PIC_CG_INNER)]
    with pytest.raises(pic.PicError) as e:
        pic.pic_init_batch(prm)
    assert e.value.code == pic.PIC_EINVAL


def test_batch_mixing_chebyshev_and_cg_simulations_matches_individual_runs():
    # a simulation asking for rtol 1e-14 takes the inner CG inside the Chebyshev-form
    # kernel; its batch neighbour (rtol 1e-12, theta 1) takes the tiles. Each gives the
    # fields it gives alone, bit for bit.
    nx, ny, ppc = 64, 64, 3
    w, sp, F0 = workload(nx, ny, ppc, gamma0=5.0, u_th=0.2, seed=21, field_amp=0.05, colocated=False)
    prm = [pic.pic_params_default(nx=nx, ny=ny, shape_order=2, gamma0=5.0, ppc=ppc, cg_rtol=rt,
                                  precision=pic.PIC_MIXED32, theta=th) for th, rt in ((0.5, 1e-14), (1.0, 1e-12))]

    def run(params, k):
        h = pic.pic_init_batch(params) if len(params) > 1 else pic.pic_init(params[0])
        try:
            for q in range(len(params)):
                if len(params) > 1:
                    pic.pic_select(h, q)
                for c in range(6):
                    pic.pic_set_fields(h, c, np.ascontiguousarray(F0[c]).ravel())
                for s, d in enumerate(sp):
                    pic.pic_load_particles(h, s, d["x"], d["y"], d["ux"], d["uy"], d["uz"])
            pic.pic_step(h, 3)
            if len(params) > 1:
                pic.pic_select(h, k)
            m = pic.pic_moments(h)
            return np.stack([pic.fields_numpy(h, c, nx, ny) for c in range(12)]), m
        finally:
            pic.pic_free(h)

    for k in range(2):
        Fb, mb = run(prm, k)
        Fa, ma = run([prm[k]], 0)
        assert np.array_equal(Fb, Fa), k
        assert mb["cg_rel_resid"] <= prm[k].cg_rtol and ma["cg_iters_total"] == mb["cg_iters_total"]
