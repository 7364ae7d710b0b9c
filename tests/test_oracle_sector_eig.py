"""Pins for oracle.sector and oracle.eig: brute force, sector union, iterative vs dense."""
import numpy as np
import pytest

from oracle.hamiltonian import problem_1d, Problem, coefficients_from_masses
from oracle.sector import sector_basis, reflect_x, ANY, X_EVEN, X_ODD
from oracle.eig import (all_eigenvalues_dense, lowest_dense, lowest_iterative,
                        residual_norms, rayleigh_quotients, certify)


def test_sector_union_is_full_spectrum():
    # brute force n <= 16: the even and odd blocks together are the whole spectrum
    P = problem_1d(20.0, 1.0, 1.0, (12, 8), (4.0, 4.0), 1.0, 1.0)
    full = np.linalg.eigvalsh(P.assemble_dense())
    ev = all_eigenvalues_dense(P, X_EVEN)
    od = all_eigenvalues_dense(P, X_ODD)
    assert ev.size == (12 // 2 + 1) * 8 and od.size == (12 // 2 - 1) * 8
    both = np.sort(np.concatenate([ev, od]))
    assert np.max(np.abs(both - full)) <= 1e-12 * np.abs(full).max()
    assert np.max(np.abs(all_eigenvalues_dense(P, ANY) - full)) <= 1e-12 * np.abs(full).max()


def test_sector_basis_orthonormal_and_invariant():
    P = problem_1d(20.0, 1.0, 1.0, (10, 6), (4.0, 4.0), 1.0, 1.0)
    for parity, s in [(X_EVEN, 1.0), (X_ODD, -1.0)]:
        B = sector_basis(P, parity).toarray()
        assert np.allclose(B.T @ B, np.eye(B.shape[1]), atol=1e-14)
        assert np.allclose(reflect_x(P, B.T), s * B.T, atol=1e-14)


@pytest.mark.parametrize("parity", [X_EVEN, X_ODD])
def test_sector_eigvectors_have_parity(parity):
    P = problem_1d(20.0, 1.0, 1.0, (16, 16), (6.0, 6.0), 1.0, 1.0)
    w, X = lowest_dense(P, 4, parity)
    s = 1.0 if parity == X_EVEN else -1.0
    assert np.max(np.abs(reflect_x(P, X) - s * X)) <= 1e-12
    res = residual_norms(P, X, w)
    assert np.max(res) <= 1e-12 * P.norm_estimate()
    assert np.allclose(rayleigh_quotients(P, X), w, rtol=0, atol=1e-13 * P.norm_estimate())


def test_iterative_matches_dense():
    P = problem_1d(20.0, 1.0, 1.0, (32, 32), (10.0, 10.0), 1.0, 1.0)
    wd, Xd = lowest_dense(P, 4, X_EVEN)
    wi, Xi = lowest_iterative(P, 4, X_EVEN, tol=1e-12)
    assert np.max(np.abs(wi - wd) / np.abs(wd)) <= 1e-10
    # eigenvectors agree up to sign
    for a, b in zip(Xd, Xi):
        assert min(np.linalg.norm(a - b), np.linalg.norm(a + b)) <= 1e-7


def test_certificates():
    P = problem_1d(20.0, 1.0, 1.0, (16, 12), (6.0, 6.0), 1.0, 1.0)
    spec = all_eigenvalues_dense(P, X_EVEN)
    w, X = lowest_dense(P, 3, X_EVEN)
    Xp = X + 1e-6 * np.random.default_rng(0).standard_normal(X.shape)
    th = rayleigh_quotients(P, Xp)
    res = residual_norms(P, Xp, th)
    weyl, kt = certify(th, res, spec)
    assert np.all(np.abs(th - w) <= weyl)
    assert np.all(np.abs(th - w) <= kt * 1.0000001)
    assert np.all(kt < weyl)


def test_variational_monotone_constant_potential():
    # for V = const the Fourier grids are nested in exact arithmetic only through
    # the closed form; the lowest level c is reached on every grid
    ax, ay, _ = coefficients_from_masses(20.0, 1.0, 1.0)
    for n in (8, 16):
        P = Problem((ax, ay), (n, n), (5.0, 5.0), np.full((n, n), -1.0))
        assert all_eigenvalues_dense(P, X_EVEN)[0] == pytest.approx(-1.0, abs=1e-13)
