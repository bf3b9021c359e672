"""pic_field_solve_noalloc, the allocation-free field solve, against the solve that
pic_step performs, through the C ABI.

Callers whose device memory belongs entirely to another allocator, or that must not
allocate once running, use this entry point instead of a handle. Here each call takes
the fields at the start of a pic_step and the current that step deposited, and its dB
must equal the dB that step solved for (pic_fields PIC_DBX..PIC_DBZ) to the FP64 parity
tolerance of the other tests (1e-12 relative), on two calls in a row (the scratch array
keeps the previous call's contents). The file sorts last so that a run stopping at the
first failure has already run every other test; it also passes on its own."""
import numpy as np
import pytest

import paper_1412_2480_gb300 as pic
from runners import rel, workload

pytestmark = pytest.mark.gpu


def test_noalloc_solve_matches_pic_step_on_two_calls():
    import torch
    nx, ny, ppc, cfl, theta, rtol = 96, 64, 2, 0.9, 0.6, 1e-12
    w, sp, F0 = workload(nx, ny, ppc, gamma0=3.0, u_th=0.3, seed=21, field_amp=0.05,
                         colocated=False)
    prm = pic.pic_params_default(nx=nx, ny=ny, ppc=ppc, gamma0=3.0, shape_order=2, cfl=cfl,
                                 theta=theta, cg_rtol=rtol)
    h = pic.pic_init(prm)
    try:
        for c in range(6):
            pic.pic_set_fields(h, c, np.ascontiguousarray(F0[c]).ravel())
        for s in range(2):
            d = sp[s]
            pic.pic_load_particles(h, s, d["x"], d["y"], d["ux"], d["uy"], d["uz"])
        for call in range(2):
            F_start = np.stack([pic.fields_numpy(h, c, nx, ny) for c in range(6)])
            pic.pic_step(h, 1)
            J = np.stack([pic.fields_numpy(h, c, nx, ny) for c in range(6, 9)])
            dB_ref = np.stack([pic.fields_numpy(h, c, nx, ny) for c in range(9, 12)])
            iters_ref = pic.pic_moments(h)["cg_iters_last"]
            Fd = torch.tensor(F_start.ravel(), dtype=torch.float64, device="cuda")
            Jd = torch.tensor(J.ravel(), dtype=torch.float64, device="cuda")
            dBd = torch.full((3 * nx * ny,), float("nan"), dtype=torch.float64, device="cuda")
            iters, rr = pic.pic_field_solve_noalloc(nx, ny, 1.0, 1.0, cfl, theta, rtol, 200, Fd,
                                                    Jd, dBd)
            torch.cuda.synchronize()
            dB = dBd.cpu().numpy().reshape(3, ny, nx)
            assert np.all(np.isfinite(dB))
            assert rel(dB, dB_ref) < 1e-12, f"call {call}: {rel(dB, dB_ref):.2e}"
            assert iters == iters_ref and 0 < rr <= rtol
    finally:
        pic.pic_free(h)


def test_noalloc_rejects_oversize_and_host_pointers():
    import torch
    n = 8
    F = torch.zeros(6 * n * n, dtype=torch.float64, device="cuda")
    J = torch.zeros(3 * n * n, dtype=torch.float64, device="cuda")
    dB = torch.zeros(3 * n * n, dtype=torch.float64, device="cuda")
    big = 512  # 512 x 256 cells exceeds PIC_NOALLOC_MAX_CELLS
    with pytest.raises(pic.PicError) as e:
        pic.pic_field_solve_noalloc(big, 256, 1.0, 1.0, 1.0, 0.5, 1e-10, 50, F, J, dB)
    assert e.value.code == pic.PIC_EINVAL and "PIC_NOALLOC_MAX_CELLS" in str(e.value)
    with pytest.raises(pic.PicError) as e:
        pic.pic_field_solve_noalloc(n, n, 1.0, 1.0, 1.0, 0.5, 1e-10, 50, F.cpu(), J, dB)
    assert e.value.code == pic.PIC_EINVAL
    # zero fields and current: b = 0, the solve returns dB = 0 with no iterations
    dB.fill_(1.0)
    it, rr = pic.pic_field_solve_noalloc(n, n, 1.0, 1.0, 1.0, 0.5, 1e-10, 50, F, J, dB)
    assert it == 0 and rr == 0.0 and torch.count_nonzero(dB).item() == 0
