"""pic_field_solve_noalloc, the allocation-free field solve, against the solve that
pic_step performs, through the C ABI.

Callers whose device memory belongs entirely to another allocator, or that must not
allocate once running, use this entry point instead of a handle. Here each call takes
the fields at the start of a pic_step and the current that step deposited, and its dB
must equal the dB that step solved for (pic_fields PIC_DBX..PIC_DBZ) to the FP64 parity
tolerance of the other tests (1e-12 relative), on two calls in a row (the scratch array
keeps the previous call's contents). At the size limit (nx*ny = PIC_NOALLOC_MAX_CELLS,
where the solver vectors fill the scratch layout exactly) it is compared with the
oracle's right-hand side and PCG on the same fields and current. The file sorts last so
that a run stopping at the first failure has already run every other test; it also
passes on its own."""
import ctypes as C

import numpy as np
import pytest

import oracle
import paper_1412_2480_gb300 as pic
from paper_1412_2480_gb300 import inputs
from runners import check, rel, workload

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
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            iters, rr = pic.pic_field_solve_noalloc(nx, ny, 1.0, 1.0, cfl, theta, rtol, 200, Fd,
                                                    Jd, dBd)
            torch.cuda.synchronize()
            if call == 1:  # after the one-time set-up the call reserves no device memory
                assert torch.cuda.mem_get_info()[0] == free0
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
    Fb = torch.zeros(6 * big * 256, dtype=torch.float64, device="cuda")
    Jb = torch.zeros(3 * big * 256, dtype=torch.float64, device="cuda")
    dBb = torch.zeros(3 * big * 256, dtype=torch.float64, device="cuda")
    with pytest.raises(pic.PicError) as e:
        pic.pic_field_solve_noalloc(big, 256, 1.0, 1.0, 1.0, 0.5, 1e-10, 50, Fb, Jb, dBb)
    assert e.value.code == pic.PIC_EINVAL and "PIC_NOALLOC_MAX_CELLS" in str(e.value)
    with pytest.raises(pic.PicError) as e:
        pic.pic_field_solve_noalloc(n, n, 1.0, 1.0, 1.0, 0.5, 1e-10, 50, F.cpu(), J, dB)
    assert e.value.code == pic.PIC_EINVAL
    # zero fields and current: b = 0, the solve returns dB = 0 with no iterations
    dB.fill_(1.0)
    it, rr = pic.pic_field_solve_noalloc(n, n, 1.0, 1.0, 1.0, 0.5, 1e-10, 50, F, J, dB)
    assert it == 0 and rr == 0.0 and torch.count_nonzero(dB).item() == 0


@pytest.mark.parametrize("nx,ny", [(256, 256), (1024, 64)])
def test_noalloc_at_the_size_limit_matches_the_oracle(nx, ny):
    # nx*ny = PIC_NOALLOC_MAX_CELLS: the field-kernel block count and the three solver
    # vectors reach the ends of their places in the scratch array
    import torch
    assert nx * ny == pic.PIC_NOALLOC_MAX_CELLS
    cfl, theta = 1.0, 0.5
    F = inputs.random_fields(nx, ny, 0.1, seed=nx + 7)
    rng = np.random.Generator(np.random.Philox(nx + 11))
    J = rng.standard_normal((3, ny, nx)) * 0.02
    g = oracle.grid(nx, ny, cfl, theta, 1)
    b = oracle.rhs(g, F, J)
    x, it_o, rr_o = oracle.pcg(g, b, rtol=1e-14, maxit=500)
    assert rr_o <= 1e-14
    Fd = torch.tensor(F.ravel(), dtype=torch.float64, device="cuda")
    Jd = torch.tensor(J.ravel(), dtype=torch.float64, device="cuda")
    for call in range(2):
        dBd = torch.full((3 * nx * ny,), float("nan"), dtype=torch.float64, device="cuda")
        iters, rr = pic.pic_field_solve_noalloc(nx, ny, 1.0, 1.0, cfl, theta, 1e-13, 500, Fd, Jd, dBd)
        torch.cuda.synchronize()
        dB = dBd.cpu().numpy().reshape(3, ny, nx)
        assert 0 < rr <= 1e-13 and iters > 0
        for c in range(3):
            check(dB[c], x.reshape(3, ny, nx)[c], 1e-12, f"call {call}, dB {c}")


def test_noalloc_one_cell_over_the_limit_is_rejected():
    import torch
    nx, ny = 257, 256  # one column more than the 65536-cell maximum
    F = torch.zeros(6 * nx * ny, dtype=torch.float64, device="cuda")
    J = torch.zeros(3 * nx * ny, dtype=torch.float64, device="cuda")
    dB = torch.zeros(3 * nx * ny, dtype=torch.float64, device="cuda")
    with pytest.raises(pic.PicError) as e:
        pic.pic_field_solve_noalloc(nx, ny, 1.0, 1.0, 1.0, 0.5, 1e-10, 50, F, J, dB)
    assert e.value.code == pic.PIC_EINVAL and "PIC_NOALLOC_MAX_CELLS" in str(e.value)


def test_noalloc_binding_checks_lengths_and_the_library_checks_pointers():
    import torch
    n = 8
    F = torch.zeros(6 * n * n, dtype=torch.float64, device="cuda")
    J = torch.zeros(3 * n * n, dtype=torch.float64, device="cuda")
    dB = torch.zeros(3 * n * n, dtype=torch.float64, device="cuda")
    # an undersized dB (or J) never reaches the kernels
    for args in ((F, J, dB[:-1]), (F, J[:-5], dB), (F[: 3 * n * n], J, dB)):
        with pytest.raises(pic.PicError) as e:
            pic.pic_field_solve_noalloc(n, n, 1.0, 1.0, 1.0, 0.5, 1e-10, 50, *args)
        assert e.value.code == pic.PIC_EINVAL
    # the C entry point itself refuses host memory (called without the binding's checks)
    L = pic.lib()
    pic.pic_field_solve_noalloc(n, n, 1.0, 1.0, 1.0, 0.5, 1e-10, 50, F, J, dB)  # sets argtypes
    host = np.zeros(6 * n * n)
    msg = C.create_string_buffer(128)
    rc = L.pic_field_solve_noalloc(n, n, 1.0, 1.0, 1.0, 0.5, 1e-10, 50, host.ctypes.data,
                                   J.data_ptr(), dB.data_ptr(), None, None, None, msg, len(msg))
    assert rc == pic.PIC_EINVAL and b"current device" in msg.value
