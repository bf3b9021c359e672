"""Failure paths through the C ABI, made to happen without faulting or hanging the GPU.

- A bounded wait that runs out. Every wait inside the library's kernels is bounded;
  pic_set_wait_limit and pic_cnn_set_wait_limit lower the bound to one poll, so the
  cooperative PCG's grid barriers and the tensor-core completion waits give up at once.
  The call must report PIC_ETIMEOUT, and with the default bound restored the same
  handle (and a fresh one) must work again. A tensor-core wait that gave up drains its
  matrix operations in flight before it frees tensor memory, so nothing is left running.
- A non-finite value detected on the device: a NaN loaded into one node of Ex (the host
  copies fields as they are) reaches the particles through the gather; the push flags
  the non-finite momentum and the step reports PIC_ENAN (FP64 and MIXED32)."""
import numpy as np
import pytest

import paper_1412_2480_gb300 as pic
from runners import run_gpu, workload

pytestmark = pytest.mark.gpu


def _loaded(nx, ny, ppc, precision, seed, F0=None, **kw):
    w, sp, F = workload(nx, ny, ppc, gamma0=3.0, u_th=0.3, seed=seed, field_amp=0.05, colocated=False)
    if F0 is not None:
        F = F0
    prm = pic.pic_params_default(nx=nx, ny=ny, ppc=ppc, gamma0=3.0, shape_order=2, precision=precision,
                                 cg_rtol=1e-10, **kw)
    h = pic.pic_init(prm)
    for c in range(6):
        pic.pic_set_fields(h, c, np.ascontiguousarray(F[c]).ravel())
    for s, d in enumerate(sp):
        pic.pic_load_particles(h, s, d["x"], d["y"], d["ux"], d["uy"], d["uz"])
    return h


def test_cooperative_solve_barrier_timeout_is_reported_and_recoverable():
    nx, ny = 512, 256  # 64 chunks of 2048 cells: 64 CTAs meet at every grid barrier
    h = _loaded(nx, ny, 2, pic.PIC_MIXED32, seed=41)
    try:
        pic.pic_step(h, 1)
        assert pic.pic_moments(h)["cg_rel_resid"] <= 1e-10
        pic.pic_set_wait_limit(h, 1)
        with pytest.raises(pic.PicError) as e:
            pic.pic_step(h, 1)
        assert e.value.code == pic.PIC_ETIMEOUT, e.value
        assert "barrier" in str(e.value)
        pic.pic_set_wait_limit(h, 0)
        pic.pic_step(h, 2)  # the same handle goes on: the solve meets its tolerance again
        m = pic.pic_moments(h)
        assert m["step"] == 4 and 0 < m["cg_rel_resid"] <= 1e-10
        with pytest.raises(pic.PicError) as e:
            pic.pic_set_wait_limit(h, -1)
        assert e.value.code == pic.PIC_EINVAL
    finally:
        pic.pic_free(h)
    # the device is unaffected: a fresh handle runs a clean step
    w, sp, F0 = workload(64, 32, 2, gamma0=3.0, u_th=0.3, seed=42, field_amp=0.05, colocated=False)
    _, _, mom = run_gpu(64, 32, 2, sp, F0, 2, 2, gamma0=3.0, precision=pic.PIC_MIXED32)
    assert mom["step"] == 2 and mom["cg_rel_resid"] <= 1e-10


def test_tensor_core_wait_timeout_is_reported_and_recoverable():
    c = pic.pic_cnn_create()
    try:
        rng = np.random.default_rng(5)
        pic.pic_cnn_set_params(c, (rng.standard_normal(pic.PIC_CNN_NPARAMS) * 0.05).astype(np.float32))
        x = rng.standard_normal((2, 3, 64, 64)).astype(np.float32)
        t = rng.standard_normal((2, 3, 64, 64)).astype(np.float32)
        y_ref = pic.pic_cnn_forward(c, x)
        g_ref, loss_ref = pic.pic_cnn_gradient(c, x, t)
        pic.pic_cnn_set_wait_limit(c, 1)
        for call in (lambda: pic.pic_cnn_forward(c, x), lambda: pic.pic_cnn_gradient(c, x, t)):
            with pytest.raises(pic.PicError) as e:
                call()
            assert e.value.code == pic.PIC_ETIMEOUT, e.value
        pic.pic_cnn_set_wait_limit(c, 0)
        np.testing.assert_array_equal(pic.pic_cnn_forward(c, x), y_ref)
        g, loss = pic.pic_cnn_gradient(c, x, t)
        assert loss == pytest.approx(loss_ref, rel=1e-9)
        # weight gradients are summed with FP32 atomics in any order: equal to rounding
        np.testing.assert_allclose(g, g_ref, rtol=1e-4, atol=1e-6 * np.abs(g_ref).max())
    finally:
        pic.pic_cnn_free(c)


@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_MIXED32])
def test_non_finite_field_value_is_detected_on_the_device(precision):
    nx, ny, ppc = 64, 32, 2
    w, sp, F0 = workload(nx, ny, ppc, gamma0=3.0, u_th=0.3, seed=43, field_amp=0.05, colocated=False)
    F0 = F0.copy()
    F0[0][11, 17] = np.nan  # one node of Ex
    h = _loaded(nx, ny, ppc, precision, seed=43, F0=F0)
    try:
        with pytest.raises(pic.PicError) as e:
            pic.pic_step(h, 3)
        assert e.value.code == pic.PIC_ENAN, e.value
        assert pic.pic_moments(h)["step"] == 1  # the failing step completed, the rest were skipped
    finally:
        pic.pic_free(h)
