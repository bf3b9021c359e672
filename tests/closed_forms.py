"""Closed forms and independent references used to pin the oracle and the CUDA path.

Nothing here calls the oracle or the CUDA library. Every function is a textbook or
library definition, or a closed form the paper prints (Ikeya & Matsumoto, PASJ 2015):
  * the vacuum numerical dispersion relation, Eq. (10), its theta = 1/2 form Eq. (15)
    and the paper's approximate Re/Im split, Eqs. (11)-(12);
  * the spectral (Fourier) form of the operator of Eq. (7) on a periodic grid;
  * centred cardinal B-splines from scipy;
  * Yee difference operators written with numpy.roll, used to check the paper's
    time discretisation Eqs. (5)-(6) directly.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.interpolate import BSpline


def S_xy(cfl_x: float, cfl_y: float, kx: float, ky: float, dx=1.0, dy=1.0):
    """Eqs. (13)-(14): S_x = c dt/dx sin(kx dx/2), S_y likewise."""
    return cfl_x * math.sin(kx * dx / 2), cfl_y * math.sin(ky * dy / 2)


def amplification(theta: float, S: float) -> complex:
    """Root lambda = e^{i omega dt} of Eq. (10), solved for e^{i omega dt}:
    with T = (lambda - 1)/(theta (lambda - 1) + 1), Eq. (10) reads T^2 = -4 S^2, so
    T = 2iS (one branch) and lambda = (1 + 2i(1-theta)S) / (1 - 2i theta S)."""
    return (1 + 2j * (1 - theta) * S) / (1 - 2j * theta * S)


def eq10_residual(theta: float, lam: complex, Sx: float, Sy: float) -> complex:
    """Left-hand side of Eq. (10) with e^{i omega dt} = lam."""
    T = (lam - 1) / (theta * (lam - 1) + 1)
    return T * T + 4 * Sx * Sx + 4 * Sy * Sy


def eq11_real(theta: float, S: float) -> float:
    """The paper's printed Eq. (11) (approximate Re[omega dt])."""
    inv = 1.0 / (S * S)
    return 2 * math.atan(0.25 * math.sqrt(inv) / ((theta - 0.5) ** 2 + 0.25 * inv))


def eq12_imag(theta: float, S: float) -> float:
    """The paper's printed Eq. (12) (approximate Im[omega dt])."""
    inv = 1.0 / (S * S)
    return 2 * math.atan(0.5 * (theta - 0.5) / ((theta - 0.5) ** 2 + 0.25 * inv))


def bspline(p: int):
    """Centred cardinal B-spline of degree p, from scipy (knots -(p+1)/2 .. (p+1)/2)."""
    knots = np.arange(p + 2, dtype=np.float64) - (p + 1) / 2.0
    b = BSpline.basis_element(knots, extrapolate=False)

    def f(d):
        v = b(np.asarray(d, dtype=np.float64))
        return np.nan_to_num(v, nan=0.0)

    return f


def k2_symbol(nx, ny, dx=1.0, dy=1.0):
    """Fourier symbol of minus the 5-point Laplacian: 4 sin^2(kx dx/2)/dx^2 + ..."""
    kx = 2 * math.pi * np.fft.fftfreq(nx)
    ky = 2 * math.pi * np.fft.fftfreq(ny)
    KY, KX = np.meshgrid(ky, kx, indexing="ij")
    return 4 * np.sin(KX / 2) ** 2 / dx**2 + 4 * np.sin(KY / 2) ** 2 / dy**2


def spectral_solve(b3, nx, ny, theta, dt, dx=1.0, dy=1.0):
    """Direct solve of [1 - (theta dt)^2 Lap] x = b on each periodic lattice by FFT."""
    lam = 1.0 + (theta * dt) ** 2 * k2_symbol(nx, ny, dx, dy)
    out = np.empty_like(b3)
    for c in range(3):
        out[c] = np.real(np.fft.ifft2(np.fft.fft2(b3[c]) / lam))
    return out


# ---- Yee operators with numpy.roll (arrays shaped (ny, nx), axis 1 = x) --------

def _fwd(a, axis):  # a[i+1] - a[i]
    return np.roll(a, -1, axis=axis) - a


def _bwd(a, axis):  # a[i] - a[i-1]
    return a - np.roll(a, 1, axis=axis)


def curl_of_E_lattice(V, dx=1.0, dy=1.0):
    Vx, Vy, Vz = V
    return np.stack([_fwd(Vz, 0) / dy, -_fwd(Vz, 1) / dx, _fwd(Vy, 1) / dx - _fwd(Vx, 0) / dy])


def curl_of_B_lattice(V, dx=1.0, dy=1.0):
    Vx, Vy, Vz = V
    return np.stack([_bwd(Vz, 0) / dy, -_bwd(Vz, 1) / dx, _bwd(Vy, 1) / dx - _bwd(Vx, 0) / dy])


def div_nodes(V, dx=1.0, dy=1.0):
    return _bwd(V[0], 1) / dx + _bwd(V[1], 0) / dy


def relerr(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
