"""The alternative gather reading (PIC_GATHER_NODAL: E and B averaged to the nodes,
then gathered with the deposit's node weights), GPU against the oracle's nodal gather
through the C ABI: one step of a hot plasma in random fields (orders 1-3; FP64 to
1e-12, MIXED32 to 2e-5), a 60-step beam run, the readings differing from each other,
and the periodic-only validation."""
import numpy as np
import pytest

import paper_1412_2480_gb300 as pic
from runners import check, check_rows, match_particles, rel, run_gpu, run_oracle, workload

pytestmark = pytest.mark.gpu
TOL32 = 2e-5


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_MIXED32])
def test_nodal_step_matches_oracle(precision, order):
    nx, ny, ppc = 40, 24, 3
    w, sp, F0 = workload(nx, ny, ppc, gamma0=3.0, u_th=0.3, seed=140 + order, field_amp=0.05,
                         colocated=False)
    kw = {"tile_x": 16, "tile_y": 8} if precision == pic.PIC_MIXED32 else {}
    Fg, pg, _ = run_gpu(nx, ny, ppc, sp, F0, 1, order, gamma0=3.0, cg_rtol=1e-13, precision=precision,
                        flags=pic.PIC_GATHER_NODAL, **kw)
    Fo, po, _ = run_oracle(nx, ny, w, sp, F0, 1, order, cg_rtol=1e-13, gather="nodal")
    Fs, ps, _ = run_oracle(nx, ny, w, sp, F0, 1, order, cg_rtol=1e-13)
    tol = 1e-12 if precision == pic.PIC_FP64 else TOL32
    for c in range(9):
        check(Fg[c], Fo[c], tol, f"quantity {c}")
    for s in range(2):
        d = match_particles(pg[s], po[s], [nx, ny, 3.0, 3.0, 3.0])
        assert d < (1e-12 if precision == pic.PIC_FP64 else 1e-5), d
    # the two readings move the particles differently (well above the tolerance)
    assert rel(po[0][2:], ps[0][2:]) > 10 * tol


@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_MIXED32])
def test_nodal_beam_run_matches_oracle(precision):
    nx, ny, ppc, steps = 32, 16, 4, 60
    w, sp, F0 = workload(nx, ny, ppc, gamma0=20.0, u_th=1e-3, seed=150)
    kw = {"tile_x": 16, "tile_y": 8} if precision == pic.PIC_MIXED32 else {}
    Fg, pg, _ = run_gpu(nx, ny, ppc, sp, F0, steps, 2, theta=0.501, cg_rtol=1e-12, precision=precision,
                        flags=pic.PIC_GATHER_NODAL, **kw)
    Fo, po, _ = run_oracle(nx, ny, w, sp, F0, steps, 2, theta=0.501, cg_rtol=1e-12, gather="nodal")
    tol = 1e-9 if precision == pic.PIC_FP64 else 1e-3
    for c in range(6):
        assert rel(Fg[c], Fo[c]) < tol, f"field {c}: {rel(Fg[c], Fo[c]):.2e}"


def test_nodal_needs_periodic_boundaries():
    with pytest.raises(pic.PicError):
        pic.pic_init(pic.pic_params_default(flags=pic.PIC_GATHER_NODAL, bc_x=pic.PIC_BC_WALLS))
