"""The benchmark's shock workload at full size, cfg5: 8192 x 512 cells, a conducting,
reflecting wall at x = 0, a magnetised pair beam (sigma_B 0.1, gamma0 40, 1e-3 spread, 16
particles per cell per species) filling x < 4096 and fed by the moving injector, order 3,
theta 0.501, CFL 1 (67.1M particles), in the launch configuration the benchmark times
(captured step graph, the cooperative solve, autotuned tiles for MIXED32). One step, with
smooth random fields added to the beam's own (zero on the wall column, as pic_set_fields
and the oracle both set them), FP64 and MIXED32:

- the particle counts are the loaded particles plus the pairs the injector adds at the
  end of the step, and every one of those pairs (the oracle's counter-based draws) is in
  the GPU's set;
- 4096 loaded particles of each species, half of them within three cells of the wall
  (reflections among them), pushed by the oracle and found in the GPU's set;
- J on eight 16 x 16 node patches, one on the wall, one across the beam's front, the rest
  at random places in the beam, deposited by the oracle from every particle that can
  reach them;
- charge conservation of the step at every node more than five cells from the walls.

Tolerances as in the small tests: FP64 1e-12 (positions 1e-9 cells), MIXED32 2e-5 of the
scale of the summed terms (positions 1e-4 cells)."""
import math

import numpy as np
import pytest

import oracle
import paper_1412_2480_gb300 as pic
from paper_1412_2480_gb300 import inputs

pytestmark = pytest.mark.gpu

NX, NY, PPC, ORDER, GAMMA0, UTH, CFL, THETA = 8192, 512, 16, 3, 40.0, 1e-3, 1.0, 0.501
SEED, SIGMA_B, X0, INJ_SEED = 5, 0.1, 4096, 105
FIELD_AMP = 0.05
RTOL = 1e-10
NSAMPLE = 4096
PATCH, NPATCH, MARGIN = 16, 8, 5
TOL = {pic.PIC_FP64: 1e-12, pic.PIC_MIXED32: 2e-5}
POS_TOL = {pic.PIC_FP64: 1e-9, pic.PIC_MIXED32: 1e-4}


@pytest.fixture(scope="module")
def beam():
    w, sp, Fh = inputs.shock_beam(X0, NY, PPC, GAMMA0, UTH, SEED, sigma_b=SIGMA_B)
    F = np.empty((6, NY, NX))
    F[:] = Fh[:, :, -1:]  # the beam's uniform fields continue ahead of it
    F[:, :, :X0] = Fh
    F += inputs.random_fields(NX, NY, FIELD_AMP, SEED)
    F0 = oracle.wall_nodes_zeroed(F, NX, NY).reshape(6, NY, NX)
    return w, sp, F0


@pytest.fixture(scope="module")
def grid():
    return oracle.grid(NX, NY, CFL, THETA, ORDER, walls=True)


@pytest.fixture(scope="module", params=[pic.PIC_FP64, pic.PIC_MIXED32], ids=["fp64", "mixed32"])
def gpu_step(request, beam):
    w, sp, F0 = beam
    prec = request.param
    p = pic.pic_params_default(nx=NX, ny=NY, cfl=CFL, theta=THETA, shape_order=ORDER, gamma0=GAMMA0,
                               ppc=PPC, precision=prec, cg_rtol=RTOL, cg_max_iter=200,
                               bc_x=pic.PIC_BC_WALLS, inject_x0=float(X0), u_th=UTH, seed=INJ_SEED)
    if prec == pic.PIC_MIXED32:
        pic.pic_autotune_tiles([p], steps=3)  # as the benchmark picks its tiles
    h = pic.pic_init(p)
    try:
        for c in range(6):
            pic.pic_set_fields(h, c, np.ascontiguousarray(F0[c]).ravel())
        for s, d in enumerate(sp):
            pic.pic_load_particles(h, s, d["x"], d["y"], d["ux"], d["uy"], d["uz"])
        pic.pic_step(h, 1)
        F = np.stack([pic.fields_numpy(h, c, NX, NY) for c in range(9)])
        P = [pic.pic_particles(h, s) for s in range(2)]
        m = pic.pic_moments(h)
    finally:
        pic.pic_free(h)
    orders = [np.argsort(p[0], kind="stable") for p in P]  # for finding particles by x
    yield prec, F, P, m, orders


def _find(Pg, order, xs, e, pos_tol, u_tol):
    """Index in Pg of the particle matching the expected state e (5,), or -1."""
    lo = np.searchsorted(xs, e[0] - pos_tol)
    hi = np.searchsorted(xs, e[0] + pos_tol, side="right")
    if hi <= lo:
        return -1
    k = order[lo:hi]
    c = Pg[:, k]
    dy = np.abs(c[1] - e[1])
    dev = np.maximum.reduce([np.abs(c[0] - e[0]) / pos_tol, np.minimum(dy, NY - dy) / pos_tol,
                             np.abs(c[2] - e[2]) / u_tol, np.abs(c[3] - e[3]) / u_tol,
                             np.abs(c[4] - e[4]) / u_tol])
    j = int(np.argmin(dev))
    return int(k[j]) if dev[j] <= 1.0 else -1


def _find_all(Pg, order, expect, pos_tol, u_tol):
    xs = Pg[0][order]
    return np.array([_find(Pg, order, xs, expect[:, k], pos_tol, u_tol) for k in range(expect.shape[1])])


def test_shock_counts_and_injected_pairs(gpu_step, beam):
    prec, F, P, m, orders = gpu_step
    w, sp, F0 = beam
    assert m["step"] == 1 and m["cfl_violations"] == 0
    assert 0.0 < m["cg_rel_resid"] <= RTOL
    assert np.all(np.isfinite(F))
    x, y, mom = oracle.inject_pairs(0, NX, NY, CFL, X0, PPC, GAMMA0, UTH, INJ_SEED)
    n0 = sp[0]["x"].size
    assert m["n_particles"] == (n0 + x.size, n0 + x.size)
    for s in range(2):
        expect = np.stack([x, y, mom[s][0], mom[s][1], mom[s][2]])
        found = _find_all(P[s], orders[s], expect, POS_TOL[prec], TOL[prec] * GAMMA0)
        assert np.count_nonzero(found < 0) == 0, f"species {s}: injected pairs missing"
        assert np.unique(found).size == x.size


def test_shock_sampled_particles_match_oracle(gpu_step, beam, grid):
    prec, F, P, m, orders = gpu_step
    w, sp, F0 = beam
    rng = np.random.default_rng(4242)
    for s in range(2):
        d = sp[s]
        near = np.nonzero(d["x"] < 3.0)[0]
        idx = np.concatenate([rng.choice(near, NSAMPLE // 2, replace=False),
                              rng.choice(d["x"].size, NSAMPLE // 2, replace=False)])
        idx = np.unique(idx)
        x, y, ux, uy, uz = (np.ascontiguousarray(d[k][idx]) for k in ("x", "y", "ux", "uy", "uz"))
        _, bad = oracle.push_deposit(grid, F0, d["qm"], d["qm"] * w, x, y, ux, uy, uz)
        assert bad == 0
        reflected = np.count_nonzero(ux > 0)  # the beam moves in -x; reflected ones in +x
        assert reflected > 100
        expect = np.stack([x, y, ux, uy, uz])
        found = _find_all(P[s], orders[s], expect, POS_TOL[prec], TOL[prec] * GAMMA0)
        missing = np.count_nonzero(found < 0)
        assert missing == 0, f"species {s}: {missing} of {idx.size} sampled particles not found"
        assert np.unique(found).size == idx.size


def _patches():
    rng = np.random.default_rng(99)
    org = [(0, int(rng.integers(0, NY))), (X0 - PATCH // 2, NY - PATCH // 2)]  # wall; beam front
    while len(org) < NPATCH:
        org.append((int(rng.integers(MARGIN, X0 - PATCH - MARGIN)), int(rng.integers(0, NY))))
    return org


def test_shock_current_on_patches_matches_oracle(gpu_step, beam, grid):
    prec, F, P, m, _ = gpu_step
    w, sp, F0 = beam
    org = _patches()
    # every particle whose cell lies within MARGIN cells of a patch can reach its nodes
    # (with the wall, through its mirror image too: the wall patch starts at x = 0)
    cx = np.floor(sp[0]["x"]).astype(np.int64)
    cy = np.floor(sp[0]["y"]).astype(np.int64)
    sel = np.zeros(cx.size, dtype=bool)
    for X, Y in org:
        sel |= (np.abs(cx - (X + PATCH // 2)) < PATCH // 2 + MARGIN) & \
               (((cy - (Y - MARGIN)) % NY) < PATCH + 2 * MARGIN)
    J_all, J_pos = np.zeros(3 * NX * NY), np.zeros(3 * NX * NY)
    for s in range(2):
        d = sp[s]
        assert d["x"] is sp[0]["x"] and d["y"] is sp[0]["y"]  # co-located pairs
        for J in ((J_all, J_pos) if s == 0 else (J_all,)):
            x, y, ux, uy, uz = (np.ascontiguousarray(d[k][sel]) for k in ("x", "y", "ux", "uy", "uz"))
            oracle.push_deposit(grid, F0, d["qm"], d["qm"] * w, x, y, ux, uy, uz, J)
    Jo, Jp, Jg = J_all.reshape(3, NY, NX), J_pos.reshape(3, NY, NX), F[6:9]
    for X, Y in org:
        ix = X + np.arange(PATCH)
        iy = (Y + np.arange(PATCH)) % NY
        g = Jg[:, iy][:, :, ix]
        o = Jo[:, iy][:, :, ix]
        scale = np.linalg.norm(Jp[:, iy][:, :, ix])
        assert scale > 0
        err = np.linalg.norm(g - o) / scale
        assert err < TOL[prec], f"patch at ({X}, {Y}): {err:.2e}"


def _rho(grid, w, parts):
    r = np.zeros(NX * NY)
    for s, (x, y) in enumerate(parts):
        oracle.deposit_rho(grid, (1.0 if s == 0 else -1.0) * w, x, y, r)
    return r


@pytest.fixture(scope="module")
def gauss0(beam, grid):
    """div E - 4 pi rho of the initial state."""
    w, sp, F0 = beam
    return oracle.div_E(grid, F0) - 4 * math.pi * _rho(grid, w, [(d["x"], d["y"]) for d in sp])


def test_shock_step_conserves_charge_away_from_the_walls(gpu_step, beam, grid, gauss0):
    prec, F, P, m, _ = gpu_step
    w, sp, F0 = beam
    rho1 = _rho(grid, w, [(p[0], p[1]) for p in P])
    g1 = oracle.div_E(grid, F[:6]) - 4 * math.pi * rho1
    d = (g1 - gauss0).reshape(NY, NX)[:, 6:NX - 6]
    scale = 4 * math.pi * (np.abs(rho1).max() + w)
    assert np.abs(d).max() < TOL[prec] * scale
