"""Pins for oracle.grid: D2 built two independent ways, spectrum, exactness on trig modes."""
import numpy as np
import pytest

from oracle.grid import (grid_points, d2_spectral, d2_closed_form, wavenumbers,
                         real_fourier_basis, reflection_index)


@pytest.mark.parametrize("n,L", [(4, 1.0), (6, 2.5), (16, 20.0), (64, 20.0), (96, 7.0)])
def test_two_constructions_agree(n, L):
    A = d2_spectral(n, L)
    B = d2_closed_form(n, L)
    assert np.max(np.abs(A - B)) <= 1e-13 * np.max(np.abs(B))


@pytest.mark.parametrize("n,L", [(8, 3.0), (64, 20.0)])
def test_spectrum_closed_form(n, L):
    ev = np.sort(np.linalg.eigvalsh(d2_closed_form(n, L)))
    k = np.concatenate([[0], np.repeat(np.arange(1, n // 2), 2), [n // 2]])
    ref = np.sort(-(k * np.pi / L) ** 2)
    assert np.max(np.abs(ev - ref)) <= 1e-13 * np.max(np.abs(ref))
    # Nyquist eigenvalue is -(pi/h)^2 with h = 2L/n
    h = 2 * L / n
    assert abs(ev[0] + (np.pi / h) ** 2) <= 1e-12 * (np.pi / h) ** 2


def test_symmetric_rows_sum_zero():
    D = d2_closed_form(32, 5.0)
    assert np.allclose(D, D.T, rtol=0, atol=1e-13 * np.abs(D).max())
    assert np.max(np.abs(D.sum(axis=1))) <= 1e-12 * np.abs(D).max()


@pytest.mark.parametrize("k", [0, 1, 5, 15])
def test_exact_on_trig_modes(k):
    # the interpolant of cos/sin(k pi x/L + phi) with k < n/2 is the function itself
    n, L = 32, 4.0
    x = grid_points(n, L)
    f = np.cos(k * np.pi * x / L + 0.3)
    d2f = -(k * np.pi / L) ** 2 * f
    assert np.max(np.abs(d2_closed_form(n, L) @ f - d2f)) <= 1e-12 * max(1.0, (k * np.pi / L) ** 2)


def test_nyquist_mode():
    n, L = 16, 3.0
    h = 2 * L / n
    v = (-1.0) ** np.arange(n)
    assert np.allclose(d2_closed_form(n, L) @ v, -(np.pi / h) ** 2 * v, rtol=1e-12, atol=0)


def test_fourier_basis_orthonormal_and_grid_reflection():
    S = real_fourier_basis(12)
    assert np.allclose(S.T @ S, np.eye(12), atol=1e-14)
    assert wavenumbers(12, 1.0).size == 12
    x = grid_points(10, 2.0)
    r = reflection_index(10)
    xr = x[r]
    # x_j -> -x_j on the periodic grid (x_0 = -L is its own image, -(-L) = L == -L mod 2L)
    assert np.allclose(np.mod(xr + 2.0, 4.0), np.mod(-x + 2.0, 4.0), atol=1e-14)
    with pytest.raises(ValueError):
        grid_points(7, 1.0)
