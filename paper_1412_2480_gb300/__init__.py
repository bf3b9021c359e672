"""Python binding of the GB300 implicit-FDTD PIC library (C ABI in include/pic.h).

Argument marshalling only: every function forwards to the function of the same name in
libpic.so, which runs all of the particle cycle in CUDA kernels. Arrays may be numpy
arrays (host) or torch tensors (host or CUDA); FP64, C-contiguous. Nonzero return codes
raise PicError carrying pic_last_error(). There is no CPU fallback: if libpic.so is not
built, importing succeeds but the first call raises.

Build with ``python -c "import __graft_entry__ as g; g.build()"`` from the repository root
(or ``python paper_1412_2480_gb300/build.py``).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_HERE, "libpic.so")

PIC_OK = 0
PIC_EINVAL = -1
PIC_ENOMEM = -2
PIC_ECUDA = -3
PIC_ECG_NOCONV = -4
PIC_ECFL = -5
PIC_ENAN = -6
PIC_ETIMEOUT = -7
PIC_ESTATE = -8
PIC_FP64 = 0
PIC_MIXED32 = 1
PIC_WS_ZERO = 0
PIC_WS_PREV = 1
PIC_WS_LEARNED = 2
PIC_CNN_NPARAMS = 20259
PIC_NO_DEPOSIT = 1
PIC_NO_GRAPH = 2
PIC_NO_COOP = 4
PIC_EXPLICIT = 8
PIC_GATHER_NODAL = 16
PIC_CG_INNER = 32
PIC_BC_PERIODIC = 0
PIC_BC_WALLS = 1
PIC_EX, PIC_EY, PIC_EZ, PIC_BX, PIC_BY, PIC_BZ = range(6)
PIC_JX, PIC_JY, PIC_JZ, PIC_DBX, PIC_DBY, PIC_DBZ = range(6, 12)
PIC_RHSX, PIC_RHSY, PIC_RHSZ = range(12, 15)
PIC_RHO = 15
PIC_DENSITY_P, PIC_DENSITY_E = 16, 17

EXPORTED = ("pic_params_default", "pic_init", "pic_init_batch", "pic_select", "pic_batch_size",
            "pic_autotune_tiles", "pic_set_stream", "pic_load_particles", "pic_set_fields",
            "pic_step", "pic_profile", "pic_fields", "pic_moments", "pic_particle_count",
            "pic_particles", "pic_field_solve_noalloc", "pic_last_error", "pic_free",
            "pic_cnn_create", "pic_cnn_free", "pic_cnn_last_error", "pic_cnn_set_params",
            "pic_cnn_get_params", "pic_cnn_forward", "pic_cnn_gradient", "pic_cnn_train_step",
            "pic_cnn_stencil", "pic_set_cnn", "pic_tc_gemm_bf16", "pic_dword_check", "pic_conservation", "pic_save",
            "pic_restore", "pic_spectrum", "pic_resonance_ky", "pic_set_wait_limit",
            "pic_cnn_set_wait_limit")


class pic_params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("dx", C.c_double), ("dy", C.c_double),
                ("cfl", C.c_double), ("theta", C.c_double), ("shape_order", C.c_int32),
                ("gamma0", C.c_double), ("ppc", C.c_int32), ("skin_depth", C.c_double),
                ("precision", C.c_int32), ("cg_rtol", C.c_double), ("cg_max_iter", C.c_int32),
                ("warm_start", C.c_int32), ("flags", C.c_int32), ("tile_x", C.c_int32),
                ("tile_y", C.c_int32), ("bin_slack", C.c_double), ("bc_x", C.c_int32),
                ("inject_x0", C.c_double), ("u_th", C.c_double), ("seed", C.c_uint64)]


class pic_moments_t(C.Structure):
    _fields_ = [("step", C.c_int64), ("time", C.c_double), ("U_E", C.c_double),
                ("U_B", C.c_double), ("U_K", C.c_double), ("macro_weight", C.c_double),
                ("n_particles", C.c_int64 * 2), ("cg_iters_last", C.c_int32),
                ("cg_iters_max", C.c_int32), ("cg_iters_total", C.c_int64),
                ("cg_rel_resid", C.c_double), ("cfl_violations", C.c_int64),
                ("overflow_moves", C.c_int64), ("rebins", C.c_int64),
                ("cg_refinements", C.c_int64), ("loop_iters", C.c_int64),
                ("loop_refinements", C.c_int64), ("kernel_launches", C.c_int64)]


class PicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pic error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def lib():
    """Load libpic.so (the CUDA product). Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIBPATH):
                raise RuntimeError(f"{LIBPATH} is not built; the CUDA library is required "
                                   "(run __graft_entry__.build())")
            L = C.CDLL(LIBPATH)
            vp = C.c_void_p
            L.pic_params_default.argtypes = [C.POINTER(pic_params)]
            L.pic_params_default.restype = None
            L.pic_init.argtypes = [C.POINTER(pic_params), C.POINTER(vp)]
            L.pic_init_batch.argtypes = [C.POINTER(pic_params), C.c_int32, C.POINTER(vp)]
            L.pic_select.argtypes = [vp, C.c_int32]
            L.pic_batch_size.argtypes = [vp]
            L.pic_autotune_tiles.argtypes = [C.POINTER(pic_params), C.c_int32, C.c_int32,
                                             C.POINTER(C.c_double)]
            L.pic_set_stream.argtypes = [vp, vp]
            L.pic_load_particles.argtypes = [vp, C.c_int32, vp, vp, vp, vp, vp, C.c_int64]
            L.pic_set_fields.argtypes = [vp, C.c_int32, vp, C.c_size_t]
            L.pic_step.argtypes = [vp, C.c_int32]
            L.pic_fields.argtypes = [vp, C.c_int32, vp, C.c_size_t]
            L.pic_profile.argtypes = [vp, C.c_int32, C.POINTER(C.c_double), C.c_int32]
            L.pic_moments.argtypes = [vp, C.POINTER(pic_moments_t)]
            L.pic_particle_count.argtypes = [vp, C.c_int32]
            L.pic_particle_count.restype = C.c_int64
            L.pic_particles.argtypes = [vp, C.c_int32, vp, C.c_int64]
            L.pic_last_error.argtypes = [vp]
            L.pic_last_error.restype = C.c_char_p
            L.pic_free.argtypes = [vp]
            L.pic_free.restype = None
            L.pic_cnn_create.argtypes = [C.POINTER(vp)]
            L.pic_cnn_free.argtypes = [vp]
            L.pic_cnn_free.restype = None
            L.pic_cnn_last_error.argtypes = [vp]
            L.pic_cnn_last_error.restype = C.c_char_p
            L.pic_cnn_set_params.argtypes = [vp, vp, C.c_int64]
            L.pic_cnn_get_params.argtypes = [vp, vp, C.c_int64]
            L.pic_cnn_forward.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, vp, vp]
            L.pic_cnn_gradient.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, vp, vp, vp,
                                           C.POINTER(C.c_double)]
            L.pic_cnn_train_step.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, vp, vp, C.c_float,
                                             C.POINTER(C.c_double)]
            L.pic_set_cnn.argtypes = [vp, vp]
            L.pic_conservation.argtypes = [vp, C.POINTER(C.c_double), C.c_int32]
            L.pic_save.argtypes = [vp, C.c_char_p]
            L.pic_restore.argtypes = [vp, C.c_char_p]
            L.pic_spectrum.argtypes = [vp, C.c_int32, vp, C.c_size_t]
            L.pic_resonance_ky.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double,
                                           C.POINTER(C.c_double)]
            for name in ("pic_conservation", "pic_save", "pic_restore", "pic_spectrum",
                         "pic_resonance_ky"):
                getattr(L, name).restype = C.c_int
            L.pic_set_wait_limit.argtypes = [vp, C.c_int32]
            L.pic_set_wait_limit.restype = C.c_int
            L.pic_cnn_set_wait_limit.argtypes = [vp, C.c_int32]
            L.pic_cnn_set_wait_limit.restype = C.c_int
            L.pic_cnn_stencil.argtypes = [vp, vp, C.c_int64]
            L.pic_tc_gemm_bf16.argtypes = [C.c_int32, C.c_int32, C.c_int32, vp, vp, vp]
            L.pic_dword_check.argtypes = [vp, vp, C.c_int64, vp]
            L.pic_dword_check.restype = C.c_int
            for name in ("pic_cnn_create", "pic_cnn_set_params", "pic_cnn_get_params", "pic_cnn_forward",
                         "pic_cnn_gradient", "pic_cnn_train_step", "pic_set_cnn", "pic_tc_gemm_bf16",
                         "pic_cnn_stencil"):
                getattr(L, name).restype = C.c_int
            for name in ("pic_init", "pic_init_batch", "pic_select", "pic_batch_size",
                         "pic_autotune_tiles", "pic_set_stream", "pic_load_particles", "pic_set_fields",
                         "pic_step", "pic_profile", "pic_fields", "pic_moments", "pic_particles"):
                getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _check(rc, h):
    if rc != PIC_OK:
        msg = lib().pic_last_error(h)
        raise PicError(rc, msg.decode() if msg else "")
    return rc


def _ptr(a, writable=False):
    """Device or host address of a float64 C-contiguous numpy array or torch tensor."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):  # torch tensor
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("tensor must be contiguous float64")
        return a.data_ptr()
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous:
        raise TypeError("array must be a C-contiguous float64 numpy array")
    if writable and not a.flags.writeable:
        raise TypeError("output array is read-only")
    return a.ctypes.data


def _len(a):
    return a.numel() if hasattr(a, "numel") else a.size


# ---- the C ABI, one function each -------------------------------------------------

def pic_params_default(**overrides) -> pic_params:
    p = pic_params()
    lib().pic_params_default(C.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(f"pic_params has no field {k}")
        setattr(p, k, v)
    return p


def pic_init(params: pic_params) -> int:
    h = C.c_void_p()
    _check(lib().pic_init(C.byref(params), C.byref(h)), None)
    return h.value


def _param_array(params):
    arr = (pic_params * len(params))()
    for k, p in enumerate(params):
        arr[k] = p
    return arr


def pic_init_batch(params) -> int:
    """One handle holding len(params) simulations (a list of pic_params)."""
    arr = _param_array(params)
    h = C.c_void_p()
    _check(lib().pic_init_batch(arr, len(params), C.byref(h)), None)
    return h.value


def pic_select(h, k) -> None:
    _check(lib().pic_select(h, int(k)), h)


def pic_set_wait_limit(h, spins) -> None:
    """Polls a grid-barrier wait of the handle's cooperative solve makes before it gives up
    (the step then fails with PIC_ETIMEOUT); 0 restores the default (include/pic.h)."""
    _check(lib().pic_set_wait_limit(h, int(spins)), h)


def pic_batch_size(h) -> int:
    return lib().pic_batch_size(h)


def pic_autotune_tiles(params, steps=5):
    """Pick tile_x, tile_y for every set in `params` (updated in place); returns the
    tile-kernel ms per step of the chosen shape for shape orders 1, 2, 3."""
    arr = _param_array(params)
    best = (C.c_double * 3)()
    _check(lib().pic_autotune_tiles(arr, len(params), int(steps), best), None)
    for k in range(len(params)):
        params[k].tile_x = arr[k].tile_x
        params[k].tile_y = arr[k].tile_y
    return [best[0], best[1], best[2]]


def pic_set_stream(h, stream) -> None:
    """stream: torch.cuda.Stream, an integer cudaStream_t, or None (legacy default)."""
    sp = getattr(stream, "cuda_stream", stream)
    _check(lib().pic_set_stream(h, sp), h)


def pic_load_particles(h, species, x, y, ux, uy, uz) -> None:
    n = _len(x)
    for a in (y, ux, uy, uz):
        if _len(a) != n:
            raise ValueError("particle arrays must have equal length")
    _check(lib().pic_load_particles(h, species, _ptr(x), _ptr(y), _ptr(ux), _ptr(uy), _ptr(uz), n), h)


def pic_set_fields(h, which, data) -> None:
    _check(lib().pic_set_fields(h, which, _ptr(data), _len(data)), h)


def pic_step(h, n=1) -> None:
    _check(lib().pic_step(h, int(n)), h)


def pic_profile(h, n) -> dict:
    """Advance n steps with per-phase CUDA-event timing (see include/pic.h)."""
    out = (C.c_double * 5)()
    _check(lib().pic_profile(h, int(n), out, 5), h)
    return {"step_ms": out[0], "particle_ms": out[1], "push_kernel_ms": out[2],
            "field_ms": out[3], "cg_iters": out[4]}


def pic_fields(h, which, out=None, shape=None):
    """Copy one grid quantity into `out` (numpy or torch, nx*ny float64). With out=None a
    numpy array is returned, reshaped to `shape` when given."""
    if out is None:
        raise ValueError("pass out= (an array of nx*ny float64) or use fields_numpy()")
    _check(lib().pic_fields(h, which, _ptr(out, True), _len(out)), h)
    return out


def pic_moments(h) -> dict:
    m = pic_moments_t()
    _check(lib().pic_moments(h, C.byref(m)), h)
    d = {k: getattr(m, k) for k, _ in pic_moments_t._fields_}
    d["n_particles"] = (m.n_particles[0], m.n_particles[1])
    return d


def pic_particle_count(h, species) -> int:
    n = lib().pic_particle_count(h, species)
    if n < 0:
        raise PicError(PIC_EINVAL, "bad handle or species")
    return n


def pic_particles(h, species, out=None):
    """Returns (or fills) a (5, n) float64 array [x, y, ux, uy, uz]."""
    n = pic_particle_count(h, species)
    if out is None:
        out = np.empty((5, n), dtype=np.float64)
    _check(lib().pic_particles(h, species, _ptr(out, True), n), h)
    return out


def pic_conservation(h) -> dict:
    """Momentum, charge and Gauss-law residual of the selected simulation (see pic.h)."""
    out = (C.c_double * 6)()
    _check(lib().pic_conservation(h, out, 6), h)
    return {"momentum": (out[0], out[1], out[2]), "charge": out[3], "gauss_max": out[4],
            "gauss_rms": out[5]}


def pic_spectrum(h, which, nx, ny):
    """Amplitude spectrum of a grid quantity as an (ny, nx) array (see pic.h)."""
    out = np.empty((ny, nx), dtype=np.float64)
    _check(lib().pic_spectrum(h, int(which), out.ctypes.data, out.size), h)
    return out


def pic_resonance_ky(cfl_x, cfl_y, beta, kx_dx):
    """k_y dy of the numerical Cherenkov resonance line, Eq. (17), or None."""
    v = C.c_double(0.0)
    rc = lib().pic_resonance_ky(float(cfl_x), float(cfl_y), float(beta), float(kx_dx), C.byref(v))
    return v.value if rc == 0 else None


def pic_save(h, path) -> None:
    _check(lib().pic_save(h, os.fsencode(path)), h)


def pic_restore(h, path) -> None:
    _check(lib().pic_restore(h, os.fsencode(path)), h)


def pic_last_error(h) -> str:
    m = lib().pic_last_error(h)
    return m.decode() if m else ""


def pic_free(h) -> None:
    lib().pic_free(h)


PIC_NOALLOC_MAX_CELLS = 65536


def pic_field_solve_noalloc(nx, ny, dx, dy, cfl, theta, cg_rtol, cg_max_iter, F, J, dB,
                            stream=None):
    """Allocation-free field solve (see include/pic.h): F (6*nx*ny), J (3*nx*ny) and dB
    (3*nx*ny, written) are float64 CUDA tensors. Returns (PCG iterations, ||r||/||b||)."""
    L = lib()
    if not getattr(L, "_noalloc_typed", False):
        L.pic_field_solve_noalloc.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double,
                                              C.c_double, C.c_double, C.c_double, C.c_int32,
                                              C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.POINTER(C.c_int32), C.POINTER(C.c_double),
                                              C.c_void_p, C.c_char_p, C.c_size_t]
        L.pic_field_solve_noalloc.restype = C.c_int
        L._noalloc_typed = True
    # The C ABI sees bare pointers, so the lengths and the device are checked here:
    # an undersized or foreign-device buffer would be read or written out of bounds.
    try:
        import torch
        cur = torch.cuda.current_device()
    except Exception:  # no usable CUDA: the library call reports it
        torch, cur = None, None
    for name, a, n in (("F", F, 6), ("J", J, 3), ("dB", dB, 3)):
        on_dev = (torch is not None and isinstance(a, torch.Tensor) and a.is_cuda
                  and a.device.index == cur)
        if not on_dev:
            raise PicError(PIC_EINVAL, f"{name} must be a CUDA tensor on the current device")
        if _len(a) != n * int(nx) * int(ny):
            raise PicError(PIC_EINVAL, f"{name} must hold {n}*nx*ny = {n * int(nx) * int(ny)} "
                                       f"values, not {_len(a)}")
    it, rr = C.c_int32(0), C.c_double(0.0)
    msg = C.create_string_buffer(256)
    sp = getattr(stream, "cuda_stream", stream)
    rc = L.pic_field_solve_noalloc(int(nx), int(ny), float(dx), float(dy), float(cfl),
                                   float(theta), float(cg_rtol), int(cg_max_iter), _ptr(F),
                                   _ptr(J), _ptr(dB, True), C.byref(it), C.byref(rr), sp, msg,
                                   len(msg))
    if rc != PIC_OK:
        raise PicError(rc, msg.value.decode())
    return it.value, rr.value


# ---- learned warm start (include/pic.h) -----------------------------------------------

def _fptr(a, dtype, writable=False):
    """Address of a C-contiguous numpy array or torch tensor of the given dtype."""
    if hasattr(a, "data_ptr"):
        import torch
        want = {np.float32: torch.float32, np.uint16: torch.int16}[dtype]
        if a.dtype not in (want, torch.bfloat16 if dtype is np.uint16 else want) or not a.is_contiguous():
            raise TypeError(f"tensor must be contiguous {want}")
        return a.data_ptr()
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous:
        raise TypeError(f"array must be a C-contiguous {np.dtype(dtype).name} numpy array")
    if writable and not a.flags.writeable:
        raise TypeError("output array is read-only")
    return a.ctypes.data


def _ccheck(rc, c):
    if rc != PIC_OK:
        msg = lib().pic_cnn_last_error(c)
        raise PicError(rc, msg.decode() if msg else "")
    return rc


def pic_cnn_create() -> int:
    c = C.c_void_p()
    _ccheck(lib().pic_cnn_create(C.byref(c)), None)
    return c.value


def pic_cnn_free(c) -> None:
    lib().pic_cnn_free(c)


def pic_cnn_set_wait_limit(c, spins) -> None:
    """Polls of the network kernels' tensor-core completion waits (0: the default)."""
    _ccheck(lib().pic_cnn_set_wait_limit(c, int(spins)), c)


def pic_cnn_set_params(c, p) -> None:
    _ccheck(lib().pic_cnn_set_params(c, _fptr(p, np.float32), _len(p)), c)


def pic_cnn_get_params(c, out=None):
    if out is None:
        out = np.empty(PIC_CNN_NPARAMS, dtype=np.float32)
    _ccheck(lib().pic_cnn_get_params(c, _fptr(out, np.float32, True), _len(out)), c)
    return out


def _img_shape(a):
    s = tuple(a.shape)
    if len(s) != 4 or s[1] != 3:
        raise ValueError("images must have shape (nimg, 3, ny, nx)")
    return s[0], s[3], s[2]


def pic_cnn_forward(c, inp, out=None):
    """inp: (nimg, 3, ny, nx) float32 (numpy or torch); returns/fills out of the same shape."""
    nimg, nx, ny = _img_shape(inp)
    if out is None:
        out = np.empty((nimg, 3, ny, nx), dtype=np.float32)
    _ccheck(lib().pic_cnn_forward(c, nimg, nx, ny, _fptr(inp, np.float32), _fptr(out, np.float32, True)), c)
    return out


def pic_cnn_gradient(c, inp, target, grad=None):
    """Returns (grad, loss) of the mean squared error."""
    nimg, nx, ny = _img_shape(inp)
    if grad is None:
        grad = np.empty(PIC_CNN_NPARAMS, dtype=np.float32)
    loss = C.c_double(0.0)
    _ccheck(lib().pic_cnn_gradient(c, nimg, nx, ny, _fptr(inp, np.float32), _fptr(target, np.float32),
                                   _fptr(grad, np.float32, True), C.byref(loss)), c)
    return grad, loss.value


def pic_cnn_train_step(c, inp, target, lr=1e-3) -> float:
    nimg, nx, ny = _img_shape(inp)
    loss = C.c_double(0.0)
    _ccheck(lib().pic_cnn_train_step(c, nimg, nx, ny, _fptr(inp, np.float32), _fptr(target, np.float32),
                                     C.c_float(lr), C.byref(loss)), c)
    return loss.value


PIC_CNN_STENCIL = 732


def pic_cnn_stencil(c):
    """The network collapsed into one stencil: (K [3, 3, 9, 9], bias [3]) as float32."""
    out = np.empty(PIC_CNN_STENCIL, dtype=np.float32)
    _ccheck(lib().pic_cnn_stencil(c, _fptr(out, np.float32, True), PIC_CNN_STENCIL), c)
    return out[:729].reshape(3, 3, 9, 9), out[729:]


def pic_set_cnn(h, c) -> None:
    _check(lib().pic_set_cnn(h, c), h)


def pic_tc_gemm_bf16(A, B, D=None):
    """D = A B^T on the tensor cores; A (M, K) and B (N, K) uint16 BF16 bit patterns."""
    M, K = A.shape
    N = B.shape[0]
    if D is None:
        D = np.empty((M, N), dtype=np.float32)
    _ccheck(lib().pic_tc_gemm_bf16(M, N, K, _fptr(A, np.uint16), _fptr(B, np.uint16),
                                   _fptr(D, np.float32, True)), None)
    return D


def pic_dword_check(x, d):
    """The device's FP32-pair building blocks on x (float64) and d (int64), n each: an
    (n, 10) float32 array laid out as include/pic.h describes."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.int64)
    if x.shape != d.shape or x.ndim != 1:
        raise ValueError("x and d must be 1-D arrays of the same length")
    out = np.empty((x.size, 10), dtype=np.float32)
    _check(lib().pic_dword_check(x.ctypes.data, d.ctypes.data, x.size, out.ctypes.data), None)
    return out


# ---- conveniences built only from the calls above ----------------------------------

def fields_numpy(h, which, nx, ny):
    out = np.empty(nx * ny, dtype=np.float64)
    pic_fields(h, which, out)
    return out.reshape(ny, nx)
