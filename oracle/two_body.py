"""Two-body well depth from a binding energy (oracle; test infrastructure).

Sec. 2 (Eq. Schroedinger_equation_two_body): the heavy-light pair obeys
[-hbar^2/(2 mu_hl) Laplacian - v0 f(|xi|/sigma)] psi = E psi.  Sec. 5.1 fixes
the binding energy E = -E0 (E0 > 0) and solves the generalized eigenvalue
problem for the smallest depth v0:

    (T + E0) psi = v0 F psi,   T = -hbar^2/(2 mu_hl) D2,  F = diag f >= 0.

T + E0 is symmetric positive definite, so the v0 are the reciprocals of the
eigenvalues of the definite pencil (F, T + E0); the smallest positive v0 is
1 / lambda_max of the symmetric matrix F^1/2 (T + E0)^-1 F^1/2.

(T + E0)^-1 is formed from the definition of T on the periodic Fourier grid:
T = S diag(hbar^2 k^2 / (2 mu_hl)) S^T with S the orthonormal real Fourier basis
and k the grid's wavenumbers (``grid``), so each mode's 1/(k^2/(2 mu) + E0) keeps
full relative accuracy.  A Cholesky factorisation of T + E0 (the textbook
generalized solver) would lose the condition number (lambda_max(T) + E0)/E0, about
1e6 at E0 = 1e-4 on the sweep grids, i.e. 1e-10 in v0.  The largest eigenvalue of
the symmetric matrix is then taken with LAPACK (scipy.linalg.eigh).
The grid is the periodic Fourier grid of ``grid`` (1D: n points on
[-L, L); 2D: the n x n tensor grid).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sl

from .grid import grid_points, d2_closed_form, real_fourier_basis, wavenumbers
from .hamiltonian import shape_function


def _kinetic_and_shape(dim, mu_hl, hbar, sigma, shape, n, L):
    x = grid_points(n, L)
    D2 = d2_closed_form(n, L)
    if dim == 1:
        T = -(hbar ** 2) / (2.0 * mu_hl) * D2
        f = shape_function(np.abs(x) / sigma, shape)
    elif dim == 2:
        I = np.eye(n)
        T = -(hbar ** 2) / (2.0 * mu_hl) * (np.kron(D2, I) + np.kron(I, D2))
        X1, X2 = np.meshgrid(x, x, indexing="ij")
        f = shape_function(np.sqrt(X1 ** 2 + X2 ** 2).ravel() / sigma, shape)
    else:
        raise ValueError("dim must be 1 or 2")
    return T, f


def _kinetic_spectrum(mu_hl, hbar, n, L):
    """Orthonormal eigenvectors (columns) and exact eigenvalues of the 1D kinetic
    operator -hbar^2/(2 mu_hl) D2 on the Fourier grid."""
    return real_fourier_basis(n), (hbar ** 2) / (2.0 * mu_hl) * wavenumbers(n, L) ** 2


def tune_v0(E0: float, mu_hl: float, sigma: float, shape: int, n: int, L: float,
            dim: int = 1, hbar: float = 1.0) -> float:
    """Smallest well depth v0 whose two-body ground state has energy -E0."""
    if not E0 > 0:
        raise ValueError("E0 must be positive")
    if dim not in (1, 2):
        raise ValueError("dim must be 1 or 2")
    S, lam = _kinetic_spectrum(mu_hl, hbar, n, L)
    x = grid_points(n, L)
    if dim == 1:
        f = shape_function(np.abs(x) / sigma, shape)
    else:
        S = np.kron(S, S)
        lam = (lam[:, None] + lam[None, :]).ravel()
        X1, X2 = np.meshgrid(x, x, indexing="ij")
        f = shape_function(np.sqrt(X1 ** 2 + X2 ** 2).ravel() / sigma, shape)
    FS = np.sqrt(f)[:, None] * S                       # F^1/2 S
    G = (FS / (lam + E0)[None, :]) @ FS.T              # F^1/2 (T + E0)^-1 F^1/2
    w = sl.eigh(0.5 * (G + G.T), eigvals_only=True)
    return 1.0 / float(w.max())


def two_body_energy(v0: float, mu_hl: float, sigma: float, shape: int, n: int, L: float,
                    dim: int = 1, hbar: float = 1.0) -> float:
    """Lowest eigenvalue of T - v0 F on the same grid."""
    T, f = _kinetic_and_shape(dim, mu_hl, hbar, sigma, shape, n, L)
    return float(np.linalg.eigvalsh(T - v0 * np.diag(f))[0])


def tune_v0_2d_iterative(E0: float, mu_hl: float, sigma: float, shape: int, n: int, L: float,
                         hbar: float = 1.0) -> float:
    """2D depth for grids too large for the dense pencil: the largest eigenvalue of the
    symmetric operator F^1/2 (T + E0)^-1 F^1/2 by ARPACK, with (T + E0)^-1 applied through
    the Fourier eigendecomposition of the 1D factors of T = -hbar^2/(2 mu) (D2 (x) I + I (x) D2)."""
    import scipy.sparse.linalg as spla
    if not E0 > 0:
        raise ValueError("E0 must be positive")
    x = grid_points(n, L)
    S, lam = _kinetic_spectrum(mu_hl, hbar, n, L)
    den = lam[:, None] + lam[None, :] + E0
    X1, X2 = np.meshgrid(x, x, indexing="ij")
    sq = np.sqrt(shape_function(np.sqrt(X1 ** 2 + X2 ** 2) / sigma, shape))

    def op(v):
        u = sq * v.reshape(n, n)
        u = (S.T @ u @ S) / den
        return (sq * (S @ u @ S.T)).ravel()

    G = spla.LinearOperator((n * n, n * n), matvec=op, dtype=np.float64)
    w = spla.eigsh(G, k=1, which="LA", tol=1e-14, return_eigenvectors=False)
    return 1.0 / float(w[0])
