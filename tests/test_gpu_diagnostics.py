"""Diagnostics and checkpoints through the C ABI, GPU against the oracle: the node
charge density PIC_RHO (the integer-lattice B-spline deposit of the particles), the
conservation moments of pic_conservation (total momentum, total charge, Gauss's law
div E = 4 pi rho kept by the charge-conserving deposit, Sec. 2), and pic_save /
pic_restore round trips."""
import math

import numpy as np
import pytest

import oracle
import paper_1412_2480_gb300 as pic
from paper_1412_2480_gb300 import inputs
from runners import rel, workload

pytestmark = pytest.mark.gpu
TOL32 = 2e-5


def make(nx, ny, ppc, order, sp, F0, precision, walls=False, gamma0=3.0, **kw):
    if precision == pic.PIC_MIXED32:
        kw.setdefault("tile_x", 16)
        kw.setdefault("tile_y", 8)
    prm = pic.pic_params_default(nx=nx, ny=ny, shape_order=order, gamma0=gamma0, ppc=ppc,
                                 precision=precision, cg_rtol=1e-13,
                                 bc_x=pic.PIC_BC_WALLS if walls else pic.PIC_BC_PERIODIC, **kw)
    h = pic.pic_init(prm)
    if np.any(F0):
        for c in range(6):
            pic.pic_set_fields(h, c, np.ascontiguousarray(F0[c]).ravel())
    for s, d in enumerate(sp):
        pic.pic_load_particles(h, s, d["x"], d["y"], d["ux"], d["uy"], d["uz"])
    return h


def oracle_sim(nx, ny, w, sp, F0, order, walls=False):
    species = [oracle.Species(d["qm"], w, d["x"], d["y"], d["ux"], d["uy"], d["uz"]) for d in sp]
    return oracle.OracleSim(nx, ny, 1.0, 0.5, order, species, cg_rtol=1e-13, fields=F0, walls=walls)


def hot(nx, ny, ppc, seed, walls):
    w, sp, F0 = workload(nx, ny, ppc, gamma0=3.0, u_th=0.3, seed=seed, field_amp=0.05,
                         colocated=False)
    if walls:
        F0 = F0.copy()
        F0[[1, 2, 3], :, 0] = 0.0
    return w, sp, F0


def oracle_conservation(sim, walls):
    """The same moments from the oracle's particles and fields."""
    g = sim.g
    rho = sim.rho()
    mom = [sum(s.w * float(np.sum(getattr(s, c))) for s in sim.species) for c in ("ux", "uy", "uz")]
    r = (oracle.div_E(g, sim.F) - 4.0 * math.pi * rho).reshape(g.ny, g.nx)
    if walls:
        r = r[:, 1:]
    return {"momentum": tuple(mom), "charge": float(rho.sum()) * g.dx * g.dy,
            "gauss_max": float(np.abs(r).max()), "gauss_rms": float(np.sqrt(np.mean(r * r))),
            "rho": rho}


@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_MIXED32])
def test_rho_matches_oracle_deposit(precision, order, walls):
    nx, ny, ppc = 48, 24, 3
    w, sp, F0 = hot(nx, ny, ppc, 60 + order, walls)
    h = make(nx, ny, ppc, order, sp, F0, precision, walls)
    try:
        rho0 = pic.fields_numpy(h, pic.PIC_RHO, nx, ny).ravel()
        pic.pic_step(h, 3)
        rho3 = pic.fields_numpy(h, pic.PIC_RHO, nx, ny).ravel()
    finally:
        pic.pic_free(h)
    g = oracle.grid(nx, ny, 1.0, 0.5, order, walls=walls)
    ref0 = np.zeros(nx * ny)
    for d in sp:
        oracle.deposit_rho(g, d["qm"] * w, d["x"], d["y"], ref0)
    sim = oracle_sim(nx, ny, w, sp, F0, order, walls)
    sim.step(3)
    ref3 = sim.rho()
    tol = 1e-12 if precision == pic.PIC_FP64 else TOL32
    assert rel(rho0, ref0) < tol
    assert rel(rho3, ref3) < tol


@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_MIXED32])
def test_species_number_density_matches_oracle(precision, walls):
    # PIC_DENSITY_P / _E: macro-particles per unit area on the nodes, the deposit of a
    # unit charge per particle of one species
    nx, ny, ppc, order = 48, 24, 3, 2
    w, sp, F0 = hot(nx, ny, ppc, 75, walls)
    h = make(nx, ny, ppc, order, sp, F0, precision, walls)
    try:
        pic.pic_step(h, 2)
        got = [pic.fields_numpy(h, which, nx, ny).ravel() for which in (pic.PIC_DENSITY_P, pic.PIC_DENSITY_E)]
    finally:
        pic.pic_free(h)
    sim = oracle_sim(nx, ny, w, sp, F0, order, walls)
    sim.step(2)
    tol = 1e-12 if precision == pic.PIC_FP64 else TOL32
    for s in range(2):
        ref = np.zeros(nx * ny)
        oracle.deposit_rho(sim.g, 1.0, sim.species[s].x, sim.species[s].y, ref)
        assert rel(got[s], ref) < tol
        if not walls:  # every particle's weights sum to one
            assert abs(got[s].sum() - sim.species[s].n) < 1e-9 * sim.species[s].n


@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_MIXED32])
def test_conservation_moments_match_oracle(precision, walls):
    nx, ny, ppc, order, steps = 48, 24, 3, 2, 6
    w, sp, F0 = hot(nx, ny, ppc, 70, walls)
    h = make(nx, ny, ppc, order, sp, F0, precision, walls)
    try:
        pic.pic_step(h, steps)
        got = pic.pic_conservation(h)
    finally:
        pic.pic_free(h)
    sim = oracle_sim(nx, ny, w, sp, F0, order, walls)
    sim.step(steps)
    ref = oracle_conservation(sim, walls)
    tol = 1e-12 if precision == pic.PIC_FP64 else TOL32
    scale = max(abs(v) for v in ref["momentum"])
    for a, b in zip(got["momentum"], ref["momentum"]):
        assert abs(a - b) <= tol * scale
    # total charge: zero to round-off for the neutral periodic plasma; with walls the
    # part on the unstored wall node x = nx is left out. MIXED32 positions are FP32.
    qscale = w * nx * ny * ppc
    assert abs(got["charge"] - ref["charge"]) <= tol * qscale
    # random initial fields violate Gauss's law; the residual is carried along unchanged
    assert abs(got["gauss_max"] - ref["gauss_max"]) <= tol * ref["gauss_max"]
    assert abs(got["gauss_rms"] - ref["gauss_rms"]) <= tol * ref["gauss_rms"]


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_MIXED32])
def test_gauss_law_holds_from_a_neutral_start(precision, order):
    # co-located pairs with E = B = 0 satisfy div E = 4 pi rho = 0 at t = 0; the
    # charge-conserving deposit keeps the residual at round-off while the plasma moves.
    # Scale: one species' 4 pi rho = omega_pe^2 gamma0. FP64: 1e-12 of it. MIXED32 deposits
    # in FP32 (relative rounding 2^-24 per term, ppc (P+2)^2 terms per node and step), so
    # 20 steps stay below 20 * 4 * 25 * 6e-8 = 1.2e-4 of it: 2e-4 bound.
    nx, ny, ppc, steps, gamma0 = 48, 32, 4, 20, 3.0
    w, sp = inputs.drifting_pair_plasma(nx, ny, ppc, gamma0, 0.3, seed=80 + order)
    h = make(nx, ny, ppc, order, sp, np.zeros((6, ny, nx)), precision, gamma0=gamma0)
    try:
        c0 = pic.pic_conservation(h)
        pic.pic_step(h, steps)
        c1 = pic.pic_conservation(h)
        rho = pic.fields_numpy(h, pic.PIC_RHO, nx, ny)
    finally:
        pic.pic_free(h)
    s0 = 0.01 * gamma0  # omega_pe^2 gamma0 at skin depth 10
    assert c0["gauss_max"] <= 1e-14 * s0
    assert np.abs(rho).max() > 1e-3 * s0 / (4 * math.pi)  # the pairs have separated
    bound = 1e-12 if precision == pic.PIC_FP64 else 2e-4
    assert c1["gauss_max"] <= bound * s0, c1
    assert abs(c1["charge"]) <= 1e-12 * w * nx * ny * ppc


def state(h, nx, ny):
    F = np.stack([pic.fields_numpy(h, c, nx, ny) for c in (0, 1, 2, 3, 4, 5, 9, 10, 11)])
    parts = [pic.pic_particles(h, s) for s in range(2)]
    return F, parts, pic.pic_moments(h)


def sorted_particles(p):
    return p[:, np.lexsort(p[::-1])]


@pytest.mark.parametrize("case", ["periodic", "injector"])
@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_MIXED32])
def test_save_restore_round_trip(tmp_path, precision, case):
    nx, ny, ppc = 64, 16, 4
    if case == "periodic":
        w, sp, F0 = hot(nx, ny, ppc, 90, False)
        kw = {}
    else:
        w, sp, F0 = inputs.shock_beam(nx, ny, ppc, 10.0, 1e-3, seed=91, sigma_b=0.1)
        for d in sp:  # the beam behind the injector plane at x = 32
            keep = d["x"] < 32.0
            for k in ("x", "y", "ux", "uy", "uz"):
                d[k] = d[k][keep]
        kw = dict(walls=True, gamma0=10.0, inject_x0=32.0, u_th=1e-3, seed=17)
    path = str(tmp_path / "state.bin")
    h1 = make(nx, ny, ppc, 2, sp, F0, precision, **kw)
    h2 = make(nx, ny, ppc, 2, sp[:0], np.zeros((6, ny, nx)), precision, **kw)
    try:
        pic.pic_step(h1, 5)
        pic.pic_save(h1, path)
        F1, p1, m1 = state(h1, nx, ny)
        pic.pic_restore(h2, path)
        F2, p2, m2 = state(h2, nx, ny)
        assert np.array_equal(F1, F2)
        assert m1["step"] == m2["step"] == 5
        for s in range(2):
            assert p1[s].shape == p2[s].shape
            if precision == pic.PIC_FP64:
                assert np.array_equal(p1[s], p2[s])
            else:
                assert np.array_equal(sorted_particles(p1[s]), sorted_particles(p2[s]))
        # both continue alike (the injector's schedule included); only the order of
        # floating-point atomic sums may differ
        pic.pic_step(h1, 5)
        pic.pic_step(h2, 5)
        F1, p1, m1 = state(h1, nx, ny)
        F2, p2, m2 = state(h2, nx, ny)
        tol = 1e-11 if precision == pic.PIC_FP64 else 1e-5
        for c in range(6):
            assert rel(F2[c], F1[c]) < tol, c
        for s in range(2):
            assert p1[s].shape == p2[s].shape
        if case == "injector":
            assert p1[0].shape[1] > sp[0]["x"].size
    finally:
        pic.pic_free(h1)
        pic.pic_free(h2)


def test_restore_rejects_other_parameters_and_bad_files(tmp_path):
    nx, ny, ppc = 32, 16, 2
    w, sp, F0 = hot(nx, ny, ppc, 95, False)
    path = str(tmp_path / "s.bin")
    h1 = make(nx, ny, ppc, 1, sp, F0, pic.PIC_FP64)
    h2 = make(nx, ny, ppc, 2, sp[:0], np.zeros((6, ny, nx)), pic.PIC_FP64)
    h3 = make(nx, ny, ppc, 1, sp[:0], np.zeros((6, ny, nx)), pic.PIC_MIXED32)
    try:
        pic.pic_save(h1, path)
        with pytest.raises(pic.PicError):
            pic.pic_restore(h2, path)  # another shape order
        with pytest.raises(pic.PicError):
            pic.pic_restore(h3, path)  # another precision
        junk = tmp_path / "junk.bin"
        junk.write_bytes(b"not a checkpoint at all")
        with pytest.raises(pic.PicError):
            pic.pic_restore(h1, str(junk))
        short = tmp_path / "short.bin"
        short.write_bytes(open(path, "rb").read()[:200])
        with pytest.raises(pic.PicError):
            pic.pic_restore(h1, str(short))
        with pytest.raises(pic.PicError):
            pic.pic_save(h1, str(tmp_path / "no" / "such" / "dir" / "s.bin"))
        # the failed calls left the handle usable
        pic.pic_restore(h1, path)
        pic.pic_step(h1, 1)
    finally:
        for h in (h1, h2, h3):
            pic.pic_free(h)


@pytest.mark.parametrize("case", ["fp64", "mixed", "mixed_loop", "fp64_walls_injector",
                                  "mixed_walls_injector", "fp64_explicit", "mixed_explicit",
                                  "fp64_nodal", "mixed_nodal"])
def test_kernel_launch_count_graph_equals_direct(case):
    # the library counts its launches: in the step graph from its kernel nodes, in
    # direct launches from the step's structure; the two must agree (PCG loop included)
    nx, ny, ppc = 64, 16, 2
    prec = pic.PIC_FP64 if case.startswith("fp64") else pic.PIC_MIXED32
    if "injector" in case:
        w, sp, F0 = inputs.shock_beam(nx, ny, ppc, 10.0, 1e-3, seed=7, sigma_b=0.1)
        for d in sp:
            keep = d["x"] < 32.0
            for k in ("x", "y", "ux", "uy", "uz"):
                d[k] = d[k][keep]
        kw = dict(walls=True, gamma0=10.0, inject_x0=32.0, u_th=1e-3, seed=3)
    else:
        w, sp, F0 = hot(nx, ny, ppc, 97, False)
        kw = {}
    counts = []
    for flags in (0, pic.PIC_NO_GRAPH):
        if case == "mixed_loop":
            flags |= pic.PIC_NO_COOP
        if case.endswith("explicit"):
            flags |= pic.PIC_EXPLICIT
            kw["cfl"] = 0.5
        if case.endswith("nodal"):
            flags |= pic.PIC_GATHER_NODAL
        h = make(nx, ny, ppc, 2, sp, F0, prec, flags=flags, **kw)
        try:
            pic.pic_step(h, 3)
            m = pic.pic_moments(h)
            counts.append(m["kernel_launches"])
        finally:
            pic.pic_free(h)
    assert counts[0] == counts[1] >= 3 * 7, counts
