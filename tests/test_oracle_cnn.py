"""Pins of the FP64 reference of the learned warm-start network (oracle/cnn.py).

The network is not in the paper (it only changes how many PCG iterations Eq. (7)
takes); these tests pin the reference against definitions that do not depend on it:
brute-force loops, adjoint identities, exact central differences and BF16 rounding."""
import numpy as np
import pytest

from oracle import cnn


def rand_params(rng, scale=1.0):
    p = np.zeros(cnn.NPARAMS)
    for (ci, co), (wo, bo) in zip(cnn.LAYERS, cnn.offsets()):
        p[wo:bo] = rng.standard_normal(co * 9 * ci) * scale / np.sqrt(9 * ci)
        p[bo:bo + co] = rng.standard_normal(co) * 0.1
    return p


def test_parameter_count_and_layout():
    assert cnn.NPARAMS == 20259
    assert cnn.offsets()[1] == (896, 896 + 9216)


def test_conv_matches_brute_force_loops():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((2, 3, 5, 7))
    W = rng.standard_normal((4, 9, 3))
    b = rng.standard_normal(4)
    Y = cnn.conv(X, W, b)
    ny, nx = 5, 7
    for n in range(2):
        for co in range(4):
            for j in range(ny):
                for i in range(nx):
                    s = b[co]
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            tap = 3 * (dy + 1) + (dx + 1)
                            for ci in range(3):
                                s += W[co, tap, ci] * X[n, ci, (j + dy) % ny, (i + dx) % nx]
                    assert abs(Y[n, co, j, i] - s) < 1e-12


def test_impulse_response_is_the_kernel():
    W = np.arange(2 * 9 * 1, dtype=float).reshape(2, 9, 1) + 1
    X = np.zeros((1, 1, 6, 6))
    X[0, 0, 3, 2] = 1.0
    Y = cnn.conv(X, W, None)
    for tap in range(9):
        dy, dx = tap // 3 - 1, tap % 3 - 1
        # the pixel whose (dx, dy) neighbour is the impulse
        assert np.allclose(Y[0, :, 3 - dy, 2 - dx], W[:, tap, 0])


def test_input_and_weight_gradients_are_adjoints():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((2, 5, 6, 8))
    W = rng.standard_normal((3, 9, 5))
    dY = rng.standard_normal((2, 3, 6, 8))
    lhs = np.sum(cnn.conv(X, W, None) * dY)
    assert abs(lhs - np.sum(X * cnn.conv_input_grad(dY, W))) < 1e-10 * abs(lhs)
    assert abs(lhs - np.sum(W * cnn.conv_weight_grad(X, dY))) < 1e-10 * abs(lhs)


def test_gradient_equals_central_differences():
    # the loss is quadratic in every single parameter: central differences are exact
    rng = np.random.default_rng(2)
    p = rand_params(rng)
    inp = rng.standard_normal((2, 3, 8, 8))
    tgt = rng.standard_normal((2, 3, 8, 8))
    L, g = cnn.loss_and_grad(p, inp, tgt)
    idx = []
    for wo, bo in cnn.offsets():
        idx += list(rng.integers(wo, bo, 6)) + [bo]
    h = 0.37
    for k in idx:
        e = np.zeros_like(p)
        e[k] = h
        fd = (cnn.loss_and_grad(p + e, inp, tgt)[0] - cnn.loss_and_grad(p - e, inp, tgt)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-9 * max(1.0, abs(g[k])) + 1e-12, k


def test_bf16_rounding_nearest_even():
    v = np.array([1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -7, -2.5, 3.0e-3, 65504.0])
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: to even (1); 1 + 3 2^-8 ties to 1 + 2^-6
    want = np.array([1.0, 1.0, 1 + 2.0 ** -6, 1 + 2.0 ** -7, -2.5])
    assert np.array_equal(cnn.bf16(v)[:5], want)
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = rng.standard_normal(10000) * 10.0 ** rng.integers(-6, 6, 10000)
    t = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cnn.bf16(x), t)


def test_linear_network_scales_with_input_when_biases_vanish():
    rng = np.random.default_rng(4)
    p = rand_params(rng)
    for (ci, co), (wo, bo) in zip(cnn.LAYERS, cnn.offsets()):
        p[bo:bo + co] = 0.0
    x = rng.standard_normal((1, 3, 8, 8))
    assert np.allclose(cnn.forward(p, 3.0 * x), 3.0 * cnn.forward(p, x), rtol=1e-12, atol=1e-12)
