"""The benchmark's batched scan at full size: the 48 uneven simulations of the scan table
(grids 128 x 128 to 512 x 256, CFL 0.5-1.0, theta 0.5-0.75, orders 1-3, 16 particles per
cell per species, gamma0 20: 87.3M particles) in one handle, in the launch configuration
the benchmark times (one persistent launch per shape order under the captured step
graph, the cooperative solve, tiles from the autotuner). One step from the seeded plasma
of every member with smooth random fields added; three members (one of each shape order,
up to 3.1M particles) run through the oracle whole and compared: fields, currents,
momenta (each component as a sorted set), all within the MIXED32 tolerance 2e-5. The
batch's particle counts and PCG residuals are checked for all 48."""
import numpy as np
import pytest

import oracle
import paper_1412_2480_gb300 as pic
from paper_1412_2480_gb300 import inputs
from runners import check, check_rows, rel

pytestmark = pytest.mark.gpu
TOL32 = 2e-5
RTOL = 1e-10
FIELD_AMP = 0.05
CHECK = (1, 14, 47)  # 256 x 256 order 2; 384 x 256 order 3, theta 0.6; 192 x 192 order 1, CFL 1


def test_scan48_batch_members_match_oracle():
    rows = inputs.scan_table()
    assert len(rows) == 48
    data = []
    for r in rows:
        w, sp = inputs.drifting_pair_plasma(r["nx"], r["ny"], r["ppc"], r["gamma0"], r["u_th"], r["seed"])
        data.append((w, sp, inputs.random_fields(r["nx"], r["ny"], FIELD_AMP, r["seed"])))
    ps = [pic.pic_params_default(nx=r["nx"], ny=r["ny"], cfl=r["cfl"], theta=r["theta"],
                                 shape_order=r["order"], gamma0=r["gamma0"], ppc=r["ppc"],
                                 precision=pic.PIC_MIXED32, cg_rtol=RTOL, cg_max_iter=200)
          for r in rows]
    pic.pic_autotune_tiles(ps, steps=3)  # as the benchmark picks its tiles
    h = pic.pic_init_batch(ps)
    got = {}
    try:
        for k, (w, sp, F0) in enumerate(data):
            pic.pic_select(h, k)
            for c in range(6):
                pic.pic_set_fields(h, c, np.ascontiguousarray(F0[c]).ravel())
            for s, d in enumerate(sp):
                pic.pic_load_particles(h, s, d["x"], d["y"], d["ux"], d["uy"], d["uz"])
        pic.pic_step(h, 1)
        for k, r in enumerate(rows):
            pic.pic_select(h, k)
            m = pic.pic_moments(h)
            n = r["nx"] * r["ny"] * r["ppc"]
            assert m["n_particles"] == (n, n), f"simulation {k}"
            assert m["step"] == 1 and m["cfl_violations"] == 0, f"simulation {k}"
            assert 0.0 < m["cg_rel_resid"] <= RTOL, f"simulation {k}"
            if k in CHECK:
                F = np.stack([pic.fields_numpy(h, c, r["nx"], r["ny"]) for c in range(9)])
                got[k] = (F, [pic.pic_particles(h, s) for s in range(2)])
    finally:
        pic.pic_free(h)
    for k in CHECK:
        r = rows[k]
        w, sp, F0 = data[k]
        species = [oracle.Species(d["qm"], w, d["x"].copy(), d["y"].copy(), d["ux"].copy(), d["uy"].copy(),
                                  d["uz"].copy()) for d in sp]
        sim = oracle.OracleSim(r["nx"], r["ny"], r["cfl"], r["theta"], r["order"], species, cg_rtol=RTOL,
                               fields=F0)
        sim.step(1)
        Fo = np.concatenate([sim.fields(), sim.J.reshape(3, r["ny"], r["nx"])])
        Fg, Pg = got[k]
        # the co-located pairs' currents cancel to ~1e-6 of either: scale by one species'
        w1 = oracle.OracleSim(r["nx"], r["ny"], r["cfl"], r["theta"], r["order"],
                              [oracle.Species(sp[0]["qm"], w, sp[0]["x"].copy(), sp[0]["y"].copy(),
                                              sp[0]["ux"].copy(), sp[0]["uy"].copy(), sp[0]["uz"].copy())],
                              cg_rtol=RTOL, fields=F0)
        w1.push_deposit()
        j_scale = np.linalg.norm(w1.J)
        for c in range(6):
            check(Fg[c], Fo[c], TOL32, f"simulation {k}, field {c}")
        assert np.linalg.norm(Fg[6:9] - Fo[6:9]) / j_scale < TOL32, f"simulation {k}, current"
        for s in range(2):
            o = np.stack([species[s].x, species[s].y, species[s].ux, species[s].uy, species[s].uz])
            check_rows(np.sort(Pg[s][2:], axis=1), np.sort(o[2:], axis=1), TOL32, f"simulation {k}, species {s}")
