"""FP64 CPU reference of the learned warm-start network -- TEST INFRASTRUCTURE.

Only the test suite loads this module; the CUDA library never does. It restates, with
plain numpy loops over the nine taps, what the tensor-core network computes:

    four 3x3 convolutions with periodic padding and biases, channels 3 -> 32 -> 32 ->
    32 -> 3, no activation; input b / rms(b), output dB_0 / rms(b);
    loss L = mean over images, channels and pixels of (output - target)^2.

Parameters are one flat vector, layer by layer: W[cout][tap][cin] with
tap = 3 (dy + 1) + (dx + 1) for the neighbour (i + dx, j + dy), then b[cout].

With quantize=True the reference rounds to BF16 (round to nearest even) exactly where
the GPU does: the input, the weights, every hidden activation and every back-propagated
activation gradient (including the output gradient); sums stay FP64. With
quantize=False it is the exact FP64 network whose gradient the tests pin by central
finite differences: for this network the loss is quadratic in each single parameter,
so central differences are exact up to rounding for any step.
"""
from __future__ import annotations

import numpy as np

LAYERS = ((3, 32), (32, 32), (32, 32), (32, 3))
NPARAMS = sum(co * 9 * ci + co for ci, co in LAYERS)


def offsets():
    """(w_off, b_off) of each layer in the flat parameter vector."""
    out, o = [], 0
    for ci, co in LAYERS:
        out.append((o, o + co * 9 * ci))
        o += co * 9 * ci + co
    return out


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    assert p.size == NPARAMS
    res = []
    for (ci, co), (wo, bo) in zip(LAYERS, offsets()):
        res.append((p[wo:wo + co * 9 * ci].reshape(co, 9, ci), p[bo:bo + co]))
    return res


def bf16(x):
    """Round FP64 values to the nearest BF16 (ties to even), through FP32 as the GPU does
    (the GPU rounds FP32 values; FP64 -> FP32 first is exact enough that a double rounding
    cannot change the BF16 result except at exact FP32 ties, which do not occur here)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def shifted(X, tap):
    """X at the neighbour (i + dx, j + dy) of every pixel, periodic; X [..., ny, nx]."""
    dy, dx = tap // 3 - 1, tap % 3 - 1
    return np.roll(X, shift=(-dy, -dx), axis=(-2, -1))


def conv(X, W, b):
    """Y[n, co] = b[co] + sum_tap sum_ci W[co, tap, ci] X[n, ci] at the tap's neighbour."""
    Y = np.zeros((X.shape[0], W.shape[0]) + X.shape[2:])
    for tap in range(9):
        Y += np.einsum("oc,ncyx->noyx", W[:, tap, :], shifted(X, tap))
    if b is not None:
        Y += b[None, :, None, None]
    return Y


def conv_input_grad(dY, W):
    """dX[n, ci] = sum_tap sum_co W[co, tap, ci] dY[n, co] at the pixel whose tap
    neighbour is this one (the adjoint of conv)."""
    dX = np.zeros((dY.shape[0], W.shape[2]) + dY.shape[2:])
    for tap in range(9):
        dy, dx = tap // 3 - 1, tap % 3 - 1
        dX += np.einsum("oc,noyx->ncyx", W[:, tap, :], np.roll(dY, shift=(dy, dx), axis=(-2, -1)))
    return dX


def conv_weight_grad(X, dY):
    """dW[co, tap, ci] = sum_n sum_pixels dY[n, co] X[n, ci] at the tap's neighbour."""
    dW = np.zeros((dY.shape[1], 9, X.shape[1]))
    for tap in range(9):
        dW[:, tap, :] = np.einsum("noyx,ncyx->oc", dY, shifted(X, tap))
    return dW


def forward(params, inp, quantize=False, keep=False):
    q = bf16 if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    layers = unpack(params)
    X = [q(inp)]
    for k, (W, b) in enumerate(layers):
        Y = conv(X[-1], q(W), b)
        X.append(q(Y) if k < 3 else Y)
    return (X[-1], X) if keep else X[-1]


def loss_and_grad(params, inp, target, quantize=False):
    """(L, dL/dparams) of the mean squared error."""
    q = bf16 if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    layers = unpack(params)
    out, X = forward(params, inp, quantize, keep=True)
    d = out - np.asarray(target, dtype=np.float64)
    L = float(np.mean(d * d))
    grad = np.zeros(NPARAMS)
    dY = q(2.0 * d / d.size)
    for k in (3, 2, 1, 0):
        W, _ = layers[k]
        wo, bo = offsets()[k]
        grad[wo:wo + W.size] = conv_weight_grad(X[k], dY).ravel()
        grad[bo:bo + W.shape[0]] = dY.sum(axis=(0, 2, 3))
        if k:
            dY = q(conv_input_grad(dY, q(W)))
    return L, grad
