"""Steady linear mountain-wave solution on a doubly periodic domain
(test helper; no part of the method under test).

Uniform flow U along x over terrain h(x, y) in a constant-N atmosphere,
small amplitude, no rotation (Smith 1980 in its Boussinesq, non-hydrostatic
form): each horizontal Fourier mode (k, l) of the vertical velocity is
    w(k, l, z) = i k U h(k, l) exp(i m z),
    m^2 = N^2 (k^2 + l^2) / (U k)^2 - (k^2 + l^2),
with m = sign(k) sqrt(m^2) for propagating modes (energy radiates upward)
and m = i sqrt(-m^2) for evanescent ones.  The decrease of the base-state
density with height multiplies the amplitude by sqrt(rho(0) / rho(z)).
"""
from __future__ import annotations

import numpy as np


def vertical_velocity(h: np.ndarray, dx: float, dy: float, U: float, N: float, z: float,
                      density_ratio: float = 1.0) -> np.ndarray:
    """w(x, y, z) on the grid of the corner heights h (ny, nx), periodic."""
    ny, nx = h.shape
    k = 2.0 * np.pi * np.fft.fftfreq(nx, d=dx)
    l = 2.0 * np.pi * np.fft.fftfreq(ny, d=dy)
    K, L = np.meshgrid(k, l)
    K2 = K * K + L * L
    hh = np.fft.fft2(h)
    w0 = 1j * K * U * hh
    with np.errstate(divide="ignore", invalid="ignore"):
        m2 = np.where(K != 0.0, N * N * K2 / (U * K) ** 2 - K2, -K2)
    m = np.where(m2 >= 0.0, np.sign(K) * np.sqrt(np.abs(m2)), 1j * np.sqrt(np.abs(m2)))
    w = np.fft.ifft2(w0 * np.exp(1j * m * z)).real
    return w * np.sqrt(density_ratio)
