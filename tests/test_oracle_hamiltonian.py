"""Pins for oracle.hamiltonian: assembly forms agree, closed-form spectra, symmetries."""
import numpy as np
import pytest

from oracle.grid import grid_points
from oracle.hamiltonian import (Problem, problem_1d, problem_2d, coefficients_from_masses,
                                coefficients_from_alpha, pair_potential_1d, GAUSS, LORENTZ3)
from oracle.sector import reflect_x, X_EVEN, X_ODD, ANY
from oracle.eig import all_eigenvalues_dense


def test_coefficients():
    ax, ay, mu = coefficients_from_masses(20.0, 1.0, 1.0)
    assert ax == pytest.approx(-1.0 / 20.0, rel=1e-15)          # mu_x = M/2 = 10
    assert ay == pytest.approx(-41.0 / 80.0, rel=1e-15)         # mu_y = 40/41
    assert mu == pytest.approx(20.0 / 21.0, rel=1e-15)
    # heavy-light units: H_config * mu_hl equals the paper's alpha form
    bx, by = coefficients_from_alpha(20.0)
    assert ax * mu == pytest.approx(bx, rel=1e-14)
    assert ay * mu == pytest.approx(by, rel=1e-14)
    assert bx == pytest.approx(-1.0 / 21.0) and by == pytest.approx(-41.0 / 84.0)


def test_potential_definition_and_symmetry():
    x = grid_points(8, 4.0)
    y = grid_points(6, 3.0)
    V = pair_potential_1d(x, y, 0.7, 1.3, GAUSS)
    i, j = 3, 1
    ref = -0.7 * (np.exp(-((y[j] - x[i] / 2) / 1.3) ** 2) + np.exp(-((y[j] + x[i] / 2) / 1.3) ** 2))
    assert V[i, j] == pytest.approx(ref, rel=1e-15)
    VL = pair_potential_1d(x, y, 1.0, 1.0, LORENTZ3)
    assert VL[i, j] == pytest.approx(-(1 / (1 + (y[j] - x[i] / 2) ** 2) ** 3 + 1 / (1 + (y[j] + x[i] / 2) ** 2) ** 3))
    r = (-np.arange(8)) % 8
    assert np.allclose(V[r, :], V, atol=0, rtol=1e-15)           # even under x -> -x


def _rand_problem_1d(nx, ny, seed=0):
    P = problem_1d(20.0, 1.0, 1.0, (nx, ny), (5.0, 4.0), 1.0, 1.0)
    return P, np.random.default_rng(seed).uniform(-1, 1, size=(3, P.N))


def test_assembly_forms_agree_1d():
    P, psi = _rand_problem_1d(8, 6)
    H = P.assemble_dense()
    Hs = P.assemble_csr()
    ref = psi @ H.T
    assert np.max(np.abs(Hs @ psi.T - ref.T)) <= 1e-12 * np.abs(ref).max()
    assert np.max(np.abs(P.apply_kron(psi) - ref)) <= 1e-12 * np.abs(ref).max()
    rows = np.array([0, 5, 17, P.N - 1])
    assert np.max(np.abs(P.apply_rows(psi[1], rows, theta=0.3) - (ref[1] - 0.3 * psi[1])[rows])) <= 1e-12 * np.abs(ref).max()
    assert np.allclose(H, H.T, atol=1e-13 * np.abs(H).max(), rtol=0)


def test_assembly_forms_agree_2d():
    P = problem_2d(20.0, 1.0, 1.0, (4, 4, 6, 6), (3.0, 3.0, 4.0, 4.0), 2.0, 1.0)
    psi = np.random.default_rng(1).uniform(-1, 1, size=(2, P.N))
    H = P.assemble_dense()
    ref = psi @ H.T
    assert np.max(np.abs(P.apply_kron(psi) - ref)) <= 1e-12 * np.abs(ref).max()
    assert np.max(np.abs((P.assemble_csr() @ psi.T).T - ref)) <= 1e-12 * np.abs(ref).max()
    rows = np.array([0, 100, P.N - 1])
    assert np.max(np.abs(P.apply_rows(psi[0], rows) - ref[0][rows])) <= 1e-12 * np.abs(ref).max()
    # x-reflection in 2D is (x1, x2) -> (-x1, -x2).  The kinetic part commutes with it; the
    # pointwise (unwrapped) pair potential does not on the boundary lines x1 = -L, x2 = -L,
    # which the reflection maps onto themselves with the other component flipped.
    Pk = Problem(P.a, P.n, P.L, np.zeros(P.n))
    assert np.max(np.abs(reflect_x(Pk, Pk.apply_kron(psi)) - Pk.apply_kron(reflect_x(Pk, psi)))) <= 1e-12 * np.abs(ref).max()
    Vr = reflect_x(P, P.V.reshape(1, -1)).reshape(P.n)
    interior = (slice(1, None), slice(1, None))
    assert np.allclose(Vr[interior], P.V[interior], rtol=1e-14, atol=0)


def test_commutes_with_reflection_1d():
    P, psi = _rand_problem_1d(10, 8)
    a = reflect_x(P, P.apply_kron(psi))
    b = P.apply_kron(reflect_x(P, psi))
    assert np.max(np.abs(a - b)) <= 1e-12 * np.abs(a).max()


def _constant_spectrum(a, n, L, c, even_x=None):
    ks = []
    for nk, Lk in zip(n, L):
        k = np.concatenate([[0], np.repeat(np.arange(1, nk // 2), 2), [nk // 2]])
        ks.append(k * np.pi / Lk)
    if even_x is not None:
        nx = n[0]
        k = np.arange(0, nx // 2 + 1) if even_x else np.arange(1, nx // 2)
        ks[0] = k * np.pi / L[0]
    grids = np.meshgrid(*ks, indexing="ij")
    lam = c + sum(-ak * g ** 2 for ak, g in zip(a, grids))
    return np.sort(lam.ravel())


@pytest.mark.parametrize("parity", [ANY, X_EVEN, X_ODD])
def test_constant_potential_closed_form_1d(parity):
    ax, ay, _ = coefficients_from_masses(20.0, 1.0, 1.0)
    n, L = (10, 8), (3.0, 5.0)
    P = Problem((ax, ay), n, L, np.full(n, -1.0))
    ev = all_eigenvalues_dense(P, parity)
    ref = _constant_spectrum((ax, ay), n, L, -1.0,
                             even_x=None if parity == ANY else (parity == X_EVEN))
    assert ev.size == ref.size
    assert np.max(np.abs(ev - ref)) <= 1e-12 * np.abs(ref).max()


def test_constant_potential_closed_form_2d():
    ax, ay, _ = coefficients_from_masses(20.0, 1.0, 1.0)
    n, L = (4, 4, 6, 6), (2.0, 2.0, 3.0, 3.0)
    P = Problem((ax, ax, ay, ay), n, L, np.full(n, -1.0))
    ev = all_eigenvalues_dense(P, ANY)
    ref = _constant_spectrum((ax, ax, ay, ay), n, L, -1.0)
    assert np.max(np.abs(ev - ref)) <= 1e-12 * np.abs(ref).max()


def test_harmonic_oscillator_spectrum():
    # V = mu_x w_x^2 x^2/2 + mu_y w_y^2 y^2/2 with oscillator lengths 1 (w = 1/mu):
    # levels (p + 1/2) w_x + (q + 1/2) w_y; x-even <=> p even.  L = 10, n = 64.
    M, m = 20.0, 1.0
    ax, ay, _ = coefficients_from_masses(M, m, 1.0)
    mu_x, mu_y = -1 / (2 * ax), -1 / (2 * ay)
    wx, wy = 1 / mu_x, 1 / mu_y
    n, L = (64, 64), (10.0, 10.0)
    x, y = grid_points(64, 10.0), grid_points(64, 10.0)
    V = 0.5 * mu_x * wx ** 2 * x[:, None] ** 2 + 0.5 * mu_y * wy ** 2 * y[None, :] ** 2
    P = Problem((ax, ay), n, L, V)
    from oracle.eig import lowest_dense
    ev, X = lowest_dense(P, 8, X_EVEN)
    levels = sorted((p + 0.5) * wx + (q + 0.5) * wy for p in range(0, 40, 2) for q in range(10))
    assert np.max(np.abs(ev - np.array(levels[:8]))) <= 1e-11
    assert np.max(np.abs(reflect_x(P, X) - X)) <= 1e-12
