"""Pins of the oracle's alternative gather reading (fields averaged to the nodes, then
gathered with the deposit's node weights), against closed forms: B-splines of degree
p >= 2 sum a quadratic's samples to x^2 + (p+1)/12 (their variance), the hat function
to x^2 + f(1-f); averaging (l+1/2)^2 over the two neighbours adds exactly 1/4. The
staggered reading, on the same fields, gives the same value without the 1/4."""
import numpy as np
import pytest

import oracle


def quad_fields(nx, ny, c, along):
    """Component c = (staggered coordinate)^2 along x or y, the others zero."""
    off_x = {0: 0.5, 1: 0.0, 2: 0.0, 3: 0.0, 4: 0.5, 5: 0.5}[c]
    off_y = {0: 0.0, 1: 0.5, 2: 0.0, 3: 0.5, 4: 0.0, 5: 0.5}[c]
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    F = np.zeros((6, ny, nx))
    F[c] = (i + off_x) ** 2 if along == "x" else (j + off_y) ** 2
    return F, (off_x if along == "x" else off_y)


def variance_term(order, frac):
    return frac * (1 - frac) if order == 1 else (order + 1) / 12.0


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("c,along", [(0, "x"), (4, "x"), (5, "x"), (1, "y"), (3, "y"), (5, "y"), (2, "x")])
def test_nodal_gather_of_a_quadratic(order, c, along):
    nx = ny = 24
    F, off = quad_fields(nx, ny, c, along)
    rng = np.random.default_rng(order * 10 + c)
    x = rng.uniform(6.0, nx - 6.0, 50)
    y = rng.uniform(6.0, ny - 6.0, 50)
    t = x if along == "x" else y
    f = t - np.floor(t)
    g = oracle.grid(nx, ny, 0.5, 0.5, order, gather="nodal")
    got = oracle.gather(g, F.ravel(), x, y)[c]
    avg = 0.25 if off else 0.0  # the two-point average of (l +- 1/2)^2 adds 1/4
    assert np.max(np.abs(got - (t * t + avg + variance_term(order, f)))) < 1e-11
    # the staggered reading interpolates on the component's own lattice: no 1/4
    gs = oracle.grid(nx, ny, 0.5, 0.5, order)
    got_s = oracle.gather(gs, F.ravel(), x, y)[c]
    fs = (t - off) - np.floor(t - off)
    assert np.max(np.abs(got_s - (t * t + variance_term(order, fs)))) < 1e-11
    others = [k for k in range(6) if k != c]
    assert np.max(np.abs(oracle.gather(g, F.ravel(), x, y)[others])) == 0.0


@pytest.mark.parametrize("order", [1, 2, 3])
def test_nodal_and_staggered_agree_on_uniform_and_linear_fields(order):
    nx, ny = 20, 16
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    F = np.zeros((6, ny, nx))
    offs = [(0.5, 0.0), (0.0, 0.5), (0.0, 0.0), (0.0, 0.5), (0.5, 0.0), (0.5, 0.5)]
    for c, (ox, oy) in enumerate(offs):
        F[c] = 1.0 + 0.3 * c + 0.01 * (i + ox) - 0.02 * (j + oy)
    rng = np.random.default_rng(order)
    x = rng.uniform(5.0, nx - 5.0, 40)
    y = rng.uniform(5.0, ny - 5.0, 40)
    a = oracle.gather(oracle.grid(nx, ny, 0.5, 0.5, order, gather="nodal"), F.ravel(), x, y)
    b = oracle.gather(oracle.grid(nx, ny, 0.5, 0.5, order), F.ravel(), x, y)
    expect = np.stack([1.0 + 0.3 * c + 0.01 * x - 0.02 * y for c in range(6)])
    assert np.max(np.abs(a - expect)) < 1e-12
    assert np.max(np.abs(b - expect)) < 1e-12


def test_nodal_reading_needs_periodic_x():
    with pytest.raises(ValueError):
        oracle.grid(16, 16, 0.5, 0.5, 2, walls=True, gather="nodal")
