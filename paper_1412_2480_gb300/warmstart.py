"""Training driver of the learned PCG warm start (include/pic.h, PIC_WS_LEARNED).

Pairs (b, dB) of Eq. (7) come from PIC runs of the library itself (the right-hand side
and solution of every step, read back with pic_fields), scaled by rms(b); the network is
trained on the GPU by the library's own forward/backward kernels (pic_cnn_train_step).
A depends only on theta, c dt / dx and dy / dx, so a network trained on small grids of
one (CFL, theta) serves every grid size with those values.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import inputs
from . import (PIC_DBX, PIC_MIXED32, PIC_RHSX, fields_numpy, pic_cnn_create, pic_cnn_free,
               pic_cnn_set_params, pic_cnn_train_step, pic_free, pic_init, pic_load_particles,
               pic_params_default, pic_set_fields, pic_step, PIC_CNN_NPARAMS)

LAYERS = ((3, 32), (32, 32), (32, 32), (32, 3))


def init_params(seed: int = 0, scale: float = 0.5) -> np.ndarray:
    """Random weights of variance scale^2 / (9 cin) per layer, zero biases."""
    rng = np.random.default_rng(seed)
    p, o = np.zeros(PIC_CNN_NPARAMS, dtype=np.float32), 0
    for ci, co in LAYERS:
        n = co * 9 * ci
        p[o:o + n] = rng.standard_normal(n) * scale / math.sqrt(9 * ci)
        o += n + co
    return p


def generate_pairs(steps: int = 300, seeds=(11, 12), nx: int = 64, ny: int = 64, cfl: float = 1.0,
                   theta: float = 0.5, order: int = 1, ppc: int = 8, gamma0: float = 20.0,
                   u_th: float = 1e-3, field_amp: float = 1e-3):
    """(b, dB) / rms(b) of every step of MIXED32 runs of a drifting pair plasma, as two
    float32 arrays of shape (n, 3, ny, nx)."""
    B, X = [], []
    for seed in seeds:
        w, sp = inputs.drifting_pair_plasma(nx, ny, ppc, gamma0, u_th, seed)
        F0 = inputs.random_fields(nx, ny, field_amp, seed) if field_amp else None
        prm = pic_params_default(nx=nx, ny=ny, cfl=cfl, theta=theta, shape_order=order, gamma0=gamma0,
                                 ppc=ppc, precision=PIC_MIXED32, cg_rtol=1e-10)
        h = pic_init(prm)
        try:
            if F0 is not None:
                for c in range(6):
                    pic_set_fields(h, c, np.ascontiguousarray(F0[c]).ravel())
            for s, d in enumerate(sp):
                pic_load_particles(h, s, d["x"], d["y"], d["ux"], d["uy"], d["uz"])
            for _ in range(steps):
                pic_step(h, 1)
                b = np.stack([fields_numpy(h, PIC_RHSX + k, nx, ny) for k in range(3)])
                x = np.stack([fields_numpy(h, PIC_DBX + k, nx, ny) for k in range(3)])
                rms = math.sqrt(float(np.mean(b * b)))
                if rms > 0:
                    B.append(b / rms)
                    X.append(x / rms)
        finally:
            pic_free(h)
    return np.asarray(B, dtype=np.float32), np.asarray(X, dtype=np.float32)


def train(B, X, iters: int = 3000, batch: int = 8, lr: float = 2e-3, seed: int = 0):
    """A network trained on the pairs (the caller frees it with pic_cnn_free); returns
    (handle, final loss, seconds)."""
    rng = np.random.default_rng(seed)
    c = pic_cnn_create()
    t0 = time.perf_counter()
    loss = float("nan")
    try:
        pic_cnn_set_params(c, init_params(seed))
        for it in range(iters):
            k = rng.integers(0, len(B), batch)
            loss = pic_cnn_train_step(c, np.ascontiguousarray(B[k]), np.ascontiguousarray(X[k]),
                                      lr=lr if it < 2 * iters // 3 else lr * 0.15)
    except Exception:
        pic_cnn_free(c)
        raise
    return c, loss, time.perf_counter() - t0
