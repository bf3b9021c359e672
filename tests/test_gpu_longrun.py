"""2000-step runs: numerical Cherenkov growth in a cold relativistic pair beam (Sec. 3),
GPU (FP64 and MIXED32) against the oracle on the same seeded inputs.

Particle trajectories are chaotic over 2000 steps, so the comparison is on what the
paper measures: the growth rate of the magnetic energy U_B(t) and its history. Growth
rate (the paper gives no definition; this suite's reading): Gamma = (1/2) d ln U_B / dt,
fitted by least squares over the steps where U_B lies between 3x its median over the
first 5 % of the run and 0.3x its maximum. History (reading): U_B averaged over windows
of 100 steps through the growth, the peak and the onset of saturation (up to the window
that starts 100 steps after the peak's window), and the mean U_B of the saturated phase
(the last 3/4 of the run). Beyond that the beam is turbulent and two runs that differ
only in rounding order part ways window by window (measured: the FP64 GPU run, whose
arithmetic differs from the oracle's only in summation order, differs by 0.3, 0.2, 3.1,
0.5, 4.4, 0.7 and 11.8 % in the seven windows after that), so only the phase average is
compared there. Growth rate and history must agree within 5 %; the saturated mean within
10 %, since one realisation of this box fluctuates by about 5 % (the same FP64 run differs
by 4.9-6.1 %).

Workload: 32 x 32 periodic, CFL 1, theta 1/2, order 1, gamma0 = 20, u_th = 1e-3,
8 particles per cell per species, co-located pairs (config 1's physics on a quarter of
its grid, so that the oracle finishes 2000 steps in well under a minute)."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import paper_1412_2480_gb300 as pic
from paper_1412_2480_gb300 import inputs
from runners import workload

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

NX = NY = 32
PPC = 8
STEPS = 2000
DT = 1.0  # CFL 1, dx = 1


def growth_rate(ub, dt=DT):
    ub = np.asarray(ub)
    n0 = max(1, len(ub) // 20)
    lo, hi = 3.0 * np.median(ub[:n0]), 0.3 * ub.max()
    peak = int(np.argmax(ub))
    idx = [k for k in range(peak + 1) if lo <= ub[k] <= hi]
    assert len(idx) >= 10, "no growth window"
    t = np.array(idx) * dt
    slope = np.polyfit(t, np.log(ub[idx]), 1)[0]
    return 0.5 * slope


def windows(ub, w=100):
    ub = np.asarray(ub)
    return ub[: len(ub) // w * w].reshape(-1, w).mean(axis=1)


@pytest.fixture(scope="module")
def oracle_ub():
    w, sp, F0 = workload(NX, NY, PPC, gamma0=20.0, u_th=1e-3, seed=1)
    species = [oracle.Species(d["qm"], w, d["x"], d["y"], d["ux"], d["uy"], d["uz"]) for d in sp]
    sim = oracle.OracleSim(NX, NY, 1.0, 0.5, 1, species, cg_rtol=1e-10)
    ub = []
    for _ in range(STEPS):
        ub.append(sim.energies()[1])  # U_B at the time level the step starts from
        sim.step(1)
    return np.array(ub)


def gpu_ub(precision):
    w, sp, F0 = workload(NX, NY, PPC, gamma0=20.0, u_th=1e-3, seed=1)
    prm = pic.pic_params_default(nx=NX, ny=NY, shape_order=1, gamma0=20.0, ppc=PPC,
                                 precision=precision, cg_rtol=1e-10, tile_x=16, tile_y=8)
    h = pic.pic_init(prm)
    ub = []
    try:
        for s, d in enumerate(sp):
            pic.pic_load_particles(h, s, d["x"], d["y"], d["ux"], d["uy"], d["uz"])
        for _ in range(STEPS):
            pic.pic_step(h, 1)
            ub.append(pic.pic_moments(h)["U_B"])  # U_B of the level the step started from
    finally:
        pic.pic_free(h)
    return np.array(ub)


@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_MIXED32])
def test_cherenkov_growth_and_energy_history_match_oracle(oracle_ub, precision):
    ub = gpu_ub(precision)
    go, gg = growth_rate(oracle_ub), growth_rate(ub)
    end = (int(np.argmax(oracle_ub)) + 200) // 100
    wo, wg = windows(oracle_ub)[:end], windows(ub)[:end]
    hist = np.max(np.abs(wg - wo) / wo)
    sat = STEPS // 4
    mo, mg = oracle_ub[sat:].mean(), ub[sat:].mean()
    print(f"precision {precision}: growth rate GPU {gg:.5f} oracle {go:.5f} "
          f"(rel {abs(gg - go) / go:.2e}); U_B windows through saturation: max difference "
          f"{hist:.2e}; saturated mean U_B GPU {mg:.4f} oracle {mo:.4f} (rel {abs(mg - mo) / mo:.2e}); "
          f"U_B grows by {oracle_ub.max() / np.median(oracle_ub[:100]):.1e}")
    assert oracle_ub.max() > 1e3 * np.median(oracle_ub[:100])  # the instability is there
    assert go > 0
    assert abs(gg - go) <= 0.05 * go
    assert hist <= 0.05
    assert abs(mg - mo) <= 0.10 * mo


# ---- config 2's physics over 2000 steps ---------------------------------------------
# Order-2 shapes, gamma0 = 40, 1e-3 spread, 32 particles per cell per species, CFL 1,
# theta 1/2 (config 2 as written, on a 128 x 32 patch of its grid). The oracle needs a
# quarter of an hour per run here, so its record is stored: tests/golden/
# longrun_cfg2_physics.json, written by tests/golden/make_longrun.py from the oracle
# alone, with the SHA-256 of the seeded inputs (checked below, so another numpy that
# built other inputs fails loudly instead of comparing different runs) and an ensemble
# of four seeds. Same-seed comparisons: the growth rate and the 100-step windows of U_B
# through the peak and one window beyond, within 5 %. After the peak U_B decays while
# the beam is turbulent; there one realisation's mean U_B (steps 500-2000) differs from
# another seed's by 3.9 % (standard deviation over the ensemble; the four seeds span
# 9.9 %), and the GPU run, whose rounding differs, is one more realisation: its mean must
# lie within the ensemble's range widened by 5 % on each side.
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "longrun_cfg2_physics.json")


@pytest.fixture(scope="module")
def cfg2_record():
    d = json.load(open(GOLDEN))
    wl = d["workload"]
    seed = d["test_seed"]
    w, sp = inputs.drifting_pair_plasma(wl["nx"], wl["ny"], wl["ppc"], wl["gamma0"], wl["u_th"], seed)
    h = hashlib.sha256()
    for s in sp:
        for k in ("x", "y", "ux", "uy", "uz"):
            h.update(np.ascontiguousarray(s[k], dtype=np.float64).tobytes())
    assert h.hexdigest() == d["runs"][str(seed)]["input_sha256"], \
        "the seeded inputs differ from the ones the stored oracle run used (numpy version?)"
    return d, w, sp


def gpu_ub_cfg2(d, sp, precision):
    wl = d["workload"]
    prm = pic.pic_params_default(nx=wl["nx"], ny=wl["ny"], shape_order=wl["order"], gamma0=wl["gamma0"],
                                 u_th=wl["u_th"], ppc=wl["ppc"], cfl=wl["cfl"], theta=wl["theta"],
                                 precision=precision, cg_rtol=wl["cg_rtol"])
    h = pic.pic_init(prm)
    ub = []
    try:
        for s, x in enumerate(sp):
            pic.pic_load_particles(h, s, x["x"], x["y"], x["ux"], x["uy"], x["uz"])
        for _ in range(wl["steps"]):
            pic.pic_step(h, 1)
            ub.append(pic.pic_moments(h)["U_B"])  # U_B of the level the step started from
    finally:
        pic.pic_free(h)
    return np.array(ub)


@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_MIXED32])
def test_config2_physics_growth_and_history_match_oracle(cfg2_record, precision):
    d, w, sp = cfg2_record
    rec = d["runs"][str(d["test_seed"])]
    uo = np.array(rec["ub"])
    ug = gpu_ub_cfg2(d, sp, precision)
    go, gg = growth_rate(uo), growth_rate(ug)
    end = (int(np.argmax(uo)) + 200) // 100
    wo, wg = windows(uo)[:end], windows(ug)[:end]
    hist = np.max(np.abs(wg - wo) / wo)
    sat = d["workload"]["steps"] // 4
    mg = ug[sat:].mean()
    ens = [r["saturated_mean_ub"] for r in d["runs"].values()]
    print(f"precision {precision}: growth rate GPU {gg:.5f} oracle {go:.5f} (rel {abs(gg - go) / go:.2e}); "
          f"U_B windows to step {end * 100}: max difference {hist:.2e}; saturated mean GPU {mg:.2f}, "
          f"oracle ensemble {min(ens):.2f}..{max(ens):.2f}")
    assert uo.max() > 1e6 * np.median(uo[:100])  # the instability is there
    assert go > 0
    assert abs(gg - go) <= 0.05 * go
    assert hist <= 0.05
    assert 0.95 * min(ens) <= mg <= 1.05 * max(ens)
