"""The benchmark's full-size workload, cfg2: 2048 x 512 cells, shape order 2, 32 particles
per cell per species (67.1M particles), gamma0 40, 1e-3 spread, CFL 1, theta 1/2, in the
launch configuration the benchmark times (captured step graph, the cooperative solve,
autotuned tiles for MIXED32). One step from the same seeded plasma, with smooth random
fields added so that the gather matters. The oracle cannot run the whole step at this
size inside a test; it checks what it can compute one by one, and the step is held to
properties that hold at any size:

- 4096 particles of each species, pushed by the oracle's gather, Boris push and move,
  are found in the GPU's particle set (positions and momenta within the path's
  tolerance);
- the current J^{n+1/2} on eight 16 x 16 node patches (one across the periodic corner,
  the others at random places, most of them across tile seams), deposited by the oracle
  from every particle that can reach them;
- charge conservation of the whole step at every node: the change of div E - 4 pi rho
  over the step is zero to rounding (Esirkepov deposit and Eq. (6)), rho being the
  oracle's deposit of the GPU's own particles before and after;
- the PCG met its tolerance; no particle was lost or moved a cell or more.

Tolerances are those of the small tests: FP64 1e-12 (positions 1e-9 cells), MIXED32 2e-5
of the scale of the summed terms (for the current of the co-located pairs, one species'
current)."""
import math

import numpy as np
import pytest

import oracle
import paper_1412_2480_gb300 as pic
from paper_1412_2480_gb300 import inputs

pytestmark = pytest.mark.gpu

NX, NY, PPC, ORDER, GAMMA0, UTH, CFL, THETA, SEED = 2048, 512, 32, 2, 40.0, 1e-3, 1.0, 0.5, 2
FIELD_AMP = 0.05
RTOL = 1e-10
NSAMPLE = 4096
PATCH, NPATCH, MARGIN = 16, 8, 4
TOL = {pic.PIC_FP64: 1e-12, pic.PIC_MIXED32: 2e-5}
POS_TOL = {pic.PIC_FP64: 1e-9, pic.PIC_MIXED32: 1e-4}


@pytest.fixture(scope="module")
def plasma():
    w, sp = inputs.drifting_pair_plasma(NX, NY, PPC, GAMMA0, UTH, SEED)
    F0 = inputs.random_fields(NX, NY, FIELD_AMP, SEED)
    return w, sp, F0


@pytest.fixture(scope="module")
def grid():
    return oracle.grid(NX, NY, CFL, THETA, ORDER)


@pytest.fixture(scope="module", params=[pic.PIC_FP64, pic.PIC_MIXED32], ids=["fp64", "mixed32"])
def gpu_step(request, plasma):
    w, sp, F0 = plasma
    prec = request.param
    p = pic.pic_params_default(nx=NX, ny=NY, cfl=CFL, theta=THETA, shape_order=ORDER, gamma0=GAMMA0,
                               ppc=PPC, u_th=UTH, precision=prec, cg_rtol=RTOL)
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
    yield prec, F, P, m


def test_fullsize_step_health(gpu_step):
    prec, F, P, m = gpu_step
    n = NX * NY * PPC
    assert m["n_particles"] == (n, n)
    assert P[0].shape == (5, n) and P[1].shape == (5, n)
    assert m["step"] == 1 and m["cfl_violations"] == 0
    assert 0.0 < m["cg_rel_resid"] <= RTOL
    assert np.all(np.isfinite(F))


def _periodic(d, L):
    d = np.abs(d)
    return np.minimum(d, L - d)


def _find(Pg, order, xs, e, pos_tol, u_tol):
    """Index in Pg of the particle matching expected state e (5,), or -1."""
    best, best_k = np.inf, -1
    for shift in (0.0, -NX, NX):
        lo = np.searchsorted(xs, e[0] + shift - pos_tol)
        hi = np.searchsorted(xs, e[0] + shift + pos_tol, side="right")
        if hi <= lo:
            continue
        k = order[lo:hi]
        c = Pg[:, k]
        dev = np.maximum.reduce([_periodic(c[0] - e[0], NX) / pos_tol, _periodic(c[1] - e[1], NY) / pos_tol,
                                 np.abs(c[2] - e[2]) / u_tol, np.abs(c[3] - e[3]) / u_tol,
                                 np.abs(c[4] - e[4]) / u_tol])
        j = int(np.argmin(dev))
        if dev[j] < best:
            best, best_k = float(dev[j]), int(k[j])
    return best_k if best <= 1.0 else -1


def test_fullsize_sampled_particles_match_oracle(gpu_step, plasma, grid):
    prec, F, P, m = gpu_step
    w, sp, F0 = plasma
    pos_tol, u_tol = POS_TOL[prec], TOL[prec] * GAMMA0
    rng = np.random.default_rng(20240)
    for s in range(2):
        d = sp[s]
        idx = rng.choice(d["x"].size, NSAMPLE, replace=False)
        x, y, ux, uy, uz = (np.ascontiguousarray(d[k][idx]) for k in ("x", "y", "ux", "uy", "uz"))
        _, bad = oracle.push_deposit(grid, F0, d["qm"], d["qm"] * w, x, y, ux, uy, uz)
        assert bad == 0
        expect = np.stack([x, y, ux, uy, uz])
        # the momentum change the fields made is well above the tolerance: the check sees
        # the gather, not only the drift
        assert np.abs(expect[2] - d["ux"][idx]).max() > 20 * u_tol
        order = np.argsort(P[s][0], kind="stable")
        xs = P[s][0][order]
        found = np.array([_find(P[s], order, xs, expect[:, k], pos_tol, u_tol) for k in range(NSAMPLE)])
        missing = np.count_nonzero(found < 0)
        assert missing == 0, f"species {s}: {missing} of {NSAMPLE} sampled particles not found"
        assert np.unique(found).size == NSAMPLE


def _patches():
    rng = np.random.default_rng(777)
    org = [(NX - PATCH // 2, NY - PATCH // 2)]  # across the periodic corner
    while len(org) < NPATCH:
        org.append((int(rng.integers(0, NX)), int(rng.integers(0, NY))))
    return org


def test_fullsize_current_on_patches_matches_oracle(gpu_step, plasma, grid):
    prec, F, P, m = gpu_step
    w, sp, F0 = plasma
    org = _patches()
    # every particle whose cell lies within MARGIN cells of a patch can reach its nodes
    cx = np.floor(sp[0]["x"]).astype(np.int64)
    cy = np.floor(sp[0]["y"]).astype(np.int64)
    J_all, J_pos = np.zeros(3 * NX * NY), np.zeros(3 * NX * NY)
    for s in range(2):
        d = sp[s]
        if s == 1 and not (d["x"] is sp[0]["x"] and d["y"] is sp[0]["y"]):
            cx = np.floor(d["x"]).astype(np.int64)
            cy = np.floor(d["y"]).astype(np.int64)
        sel = np.zeros(d["x"].size, dtype=bool)
        for X0, Y0 in org:
            sel |= (((cx - (X0 - MARGIN)) % NX) < PATCH + 2 * MARGIN) & \
                   (((cy - (Y0 - MARGIN)) % NY) < PATCH + 2 * MARGIN)
        for J in ((J_all, J_pos) if s == 0 else (J_all,)):
            x, y, ux, uy, uz = (np.ascontiguousarray(d[k][sel]) for k in ("x", "y", "ux", "uy", "uz"))
            oracle.push_deposit(grid, F0, d["qm"], d["qm"] * w, x, y, ux, uy, uz, J)
    Jo, Jp, Jg = J_all.reshape(3, NY, NX), J_pos.reshape(3, NY, NX), F[6:9]
    for X0, Y0 in org:
        ix = (X0 + np.arange(PATCH)) % NX
        iy = (Y0 + np.arange(PATCH)) % NY
        g = Jg[:, iy][:, :, ix]
        o = Jo[:, iy][:, :, ix]
        scale = np.linalg.norm(Jp[:, iy][:, :, ix])
        assert scale > 0
        err = np.linalg.norm(g - o) / scale
        assert err < TOL[prec], f"patch at ({X0}, {Y0}): {err:.2e}"


def _rho(grid, w, parts):
    r = np.zeros(NX * NY)
    for s, (x, y) in enumerate(parts):
        oracle.deposit_rho(grid, (1.0 if s == 0 else -1.0) * w, x, y, r)
    return r


@pytest.fixture(scope="module")
def gauss0(plasma, grid):
    """div E - 4 pi rho of the initial state."""
    w, sp, F0 = plasma
    return oracle.div_E(grid, F0) - 4 * math.pi * _rho(grid, w, [(d["x"], d["y"]) for d in sp])


def test_fullsize_step_conserves_charge(gpu_step, plasma, grid, gauss0):
    prec, F, P, m = gpu_step
    w, sp, F0 = plasma
    rho1 = _rho(grid, w, [(p[0], p[1]) for p in P])
    g0 = gauss0
    g1 = oracle.div_E(grid, F[:6]) - 4 * math.pi * rho1
    scale = 4 * math.pi * (np.abs(rho1).max() + w)
    assert np.abs(g1 - g0).max() < TOL[prec] * scale
