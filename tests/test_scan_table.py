"""The committed table of the 48-simulation parameter scan equals its generator, and spans
the scan the paper describes (CFL 0.5-1.0, Sec. 3.2; theta and shape orders 1-3, Sec. 3.3)."""
import json
import os

from paper_1412_2480_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def test_committed_table_matches_generator():
    path = os.path.join(HERE, "..", "paper_1412_2480_gb300", "scan48.json")
    assert json.load(open(path)) == inputs.scan_table()


def test_table_covers_the_scan():
    rows = inputs.scan_table()
    assert len(rows) == 48
    assert {r["cfl"] for r in rows} == set(inputs.SCAN_CFL)
    assert {r["theta"] for r in rows} == set(inputs.SCAN_THETA)
    assert {r["order"] for r in rows} == {1, 2, 3}
    assert len({(r["nx"], r["ny"]) for r in rows}) == 8
    # uneven sizes, about 2.7M cells and 87M macro-particles in all
    cells = sum(r["nx"] * r["ny"] for r in rows)
    assert 2.7e6 < cells < 2.75e6
    assert sum(2 * r["ppc"] * r["nx"] * r["ny"] for r in rows) == 2 * 16 * cells
