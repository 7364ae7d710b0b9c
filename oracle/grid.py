"""Periodic Fourier grid and second-derivative matrix (oracle; test infrastructure).

The paper discretises each Jacobi coordinate pseudospectrally (Sec. 3.1) and
only needs a dense matrix D for d^2/dx^2 per coordinate.  This build uses a
periodic Fourier grid on [-L, L): points x_j = -L + j*2L/n, j = 0..n-1, n even.

D2 is built two independent ways so that each pins the other:

* ``d2_spectral``   -- from its definition: trigonometric interpolation on the
  grid followed by exact differentiation.  The interpolant of grid data
  is expanded in the real Fourier modes cos(k t), sin(k t) (k < n/2) and the
  Nyquist cosine cos(n t / 2), t = pi (x + L) / L; differentiating twice
  multiplies mode k by -(k pi / L)^2.
* ``d2_closed_form`` -- the entry-wise closed form of the periodic sinc
  interpolant's second derivative (Trefethen, Spectral Methods in MATLAB,
  ch. 3): diagonal -pi^2/(3h^2) - 1/6, off-diagonal
  -(-1)^(i-j) / (2 sin^2((i-j)h/2)) on [0, 2pi) with h = 2pi/n, scaled by
  (pi/L)^2 for a box of length 2L.
"""
from __future__ import annotations

import numpy as np


def grid_points(n: int, L: float) -> np.ndarray:
    """x_j = -L + j * 2L / n for j = 0..n-1 (FP64)."""
    if n < 4 or n % 2:
        raise ValueError("n must be even and >= 4")
    return -L + np.arange(n, dtype=np.float64) * (2.0 * L / n)


def wavenumbers(n: int, L: float) -> np.ndarray:
    """Physical wavenumbers k*pi/L of the real modes in the order of ``real_fourier_basis``."""
    ks = [0]
    for k in range(1, n // 2):
        ks += [k, k]
    ks.append(n // 2)
    return np.array(ks, dtype=np.float64) * np.pi / L


def real_fourier_basis(n: int) -> np.ndarray:
    """Orthonormal real Fourier basis on n grid points, columns ordered
    [1, cos 1, sin 1, cos 2, sin 2, ..., cos(n/2-1), sin(n/2-1), Nyquist]."""
    j = np.arange(n, dtype=np.float64)
    cols = [np.full(n, 1.0 / np.sqrt(n))]
    for k in range(1, n // 2):
        t = 2.0 * np.pi * k * j / n
        cols.append(np.cos(t) * np.sqrt(2.0 / n))
        cols.append(np.sin(t) * np.sqrt(2.0 / n))
    cols.append(np.where(np.arange(n) % 2 == 0, 1.0, -1.0) / np.sqrt(n))
    return np.stack(cols, axis=1)


def d2_spectral(n: int, L: float) -> np.ndarray:
    """D2 = S diag(-(k pi/L)^2) S^T with S the orthonormal real Fourier basis."""
    S = real_fourier_basis(n)
    lam = -wavenumbers(n, L) ** 2
    return (S * lam[None, :]) @ S.T


def d2_closed_form(n: int, L: float) -> np.ndarray:
    """Entry-wise closed form of the periodic spectral second derivative."""
    if n < 4 or n % 2:
        raise ValueError("n must be even and >= 4")
    h = 2.0 * np.pi / n
    D = np.empty((n, n), dtype=np.float64)
    for i in range(n):
        for j in range(n):
            if i == j:
                D[i, j] = -np.pi ** 2 / (3.0 * h ** 2) - 1.0 / 6.0
            else:
                s = np.sin((i - j) * h / 2.0)
                D[i, j] = -((-1.0) ** (i - j)) / (2.0 * s * s)
    return D * (np.pi / L) ** 2


def reflection_index(n: int) -> np.ndarray:
    """Index map of x -> -x on the grid: j -> (n - j) mod n."""
    return (-np.arange(n)) % n
