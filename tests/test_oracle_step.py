"""Whole-step pins of the oracle and the golden fixtures.

* Gauss's law residual div E - 4 pi rho is constant in time to round-off (Esirkepov's
  charge conservation carried through Ampere's law, Eq. (6));
* div B stays at round-off; every displacement stays below one cell at CFL <= 1;
* total energy drifts by well under the paper's 1 % (Sec. 3.2) over a short run;
* the golden Fig. 2 table (written by tests/golden/make_golden.py from the oracle)
  follows Eq. (15) at theta = 1/2 and Eq. (10) at theta = 0.501;
* the paper's printed parameters: V = 0.9999c is Gamma ~ 70.7, not the stated 100
  (reading recorded); theta = 0.501 barely damps long waves (Sec. 5)."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from closed_forms import amplification
from paper_1412_2480_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def make_plasma_sim(nx=32, ny=16, ppc=4, gamma0=20.0, u_th=1e-3, seed=1, cfl=1.0, theta=0.5,
                    order=1, **kw):
    w, sp = inputs.drifting_pair_plasma(nx, ny, ppc, gamma0, u_th, seed)
    species = [oracle.Species(s["qm"], w, s["x"], s["y"], s["ux"], s["uy"], s["uz"]) for s in sp]
    return oracle.OracleSim(nx, ny, cfl, theta, order, species, **kw)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_gauss_law_and_div_b_preserved(order):
    sim = make_plasma_sim(order=order, u_th=0.05, gamma0=3.0, cg_rtol=1e-14, seed=order)
    g = sim.g
    gauss0 = oracle.div_E(g, sim.F) - 4 * math.pi * sim.rho()
    for _ in range(15):
        sim.step()
        assert sim.bad_moves == 0
        gauss = oracle.div_E(g, sim.F) - 4 * math.pi * sim.rho()
        scale = 4 * math.pi * np.abs(sim.rho()).max() + 1e-30
        assert np.abs(gauss - gauss0).max() < 1e-11 * max(scale, 1.0)
        assert np.abs(oracle.div_B(g, sim.F)).max() < 1e-11
    # the run is not trivial: fields grew from zero
    ue, ub, uk = sim.energies()
    assert ue > 0 and ub > 0


def test_energy_budget_short_run():
    sim = make_plasma_sim(nx=32, ny=32, ppc=8, order=2, cfl=1.0, theta=0.5, cg_rtol=1e-12)
    e0 = sum(sim.energies())
    for _ in range(20):
        sim.step()
    e1 = sum(sim.energies())
    assert abs(e1 - e0) < 1e-3 * e0


def test_colocated_pairs_start_neutral():
    sim = make_plasma_sim()
    assert np.abs(sim.rho()).max() < 1e-15


def _golden_rows():
    rows = []
    with open(os.path.join(GOLDEN, "vacuum_te_cfl05.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = line.split()
            rows.append((float(v[0]), int(v[1]), int(v[2]), np.array([float(a) for a in v[3:]])))
    return rows


def test_golden_fig2_table_follows_dispersion_relation():
    rows = _golden_rows()
    assert len(rows) == 16
    for theta, mx, my, amps in rows:
        kx, ky = 2 * math.pi * mx / 32, 2 * math.pi * my / 32
        S = 0.5 * math.hypot(math.sin(kx / 2), math.sin(ky / 2))
        n = np.arange(1, amps.size + 1)
        if theta == 0.5:
            ref = np.cos(n * 2 * math.atan(S))  # Eq. (15)
        else:
            ref = (amplification(theta, S) ** n).real  # Eq. (10)
        np.testing.assert_allclose(amps, ref, rtol=0, atol=1e-12)


def test_golden_table_reproduced_by_oracle():
    # the stored table still matches what the oracle computes now (regression)
    rows = _golden_rows()
    theta, mx, my, amps = rows[5]
    jj, ii = np.meshgrid(np.arange(32), np.arange(32), indexing="ij")
    mode = np.cos(2 * math.pi * (mx * (ii + 0.5) + my * (jj + 0.5)) / 32)
    F = np.zeros((6, 32, 32))
    F[5] = mode
    sim = oracle.OracleSim(32, 32, 0.5, theta, 2, [], cg_rtol=1e-15, fields=F)
    for n in range(amps.size):
        sim.step()
        a = np.sum(sim.fields()[5] * mode) / np.sum(mode * mode)
        assert abs(a - amps[n]) < 1e-13


def test_paper_printed_parameters():
    pv = json.load(open(os.path.join(GOLDEN, "paper_values.json")))
    pt = pv["periodic_test"]
    V = pt["flow_speed_over_c"]
    gamma_from_V = 1 / math.sqrt(1 - V * V)
    # Sec. 3 states V = 0.9999c "corresponds to" Gamma = 100; it is 70.7 (reading: the
    # benchmarked workloads state gamma0 directly, so nothing depends on it).
    assert abs(gamma_from_V - 70.71) < 0.01 and pt["bulk_lorentz_factor_stated"] == 100
    # Sec. 5: theta = 0.501 has little impact on long waves. Damping per unit time
    # (1/dt)(-ln|lambda|) at the paper's CFL scan ends and k dx <= 0.3:
    for cfl in (pv["cfl_scan"]["cfl_min"], pv["cfl_scan"]["cfl_max"]):
        for k in (0.05, 0.1, 0.3):
            S = cfl * math.sin(k / 2)
            damp = -math.log(abs(amplification(pv["optimal_theta"]["order2"], S))) / cfl
            assert 0 < damp < 1e-4
