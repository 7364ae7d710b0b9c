"""Two-body well depth from a binding energy (oracle; test infrastructure).

Sec. 2 (Eq. Schroedinger_equation_two_body): the heavy-light pair obeys
[-hbar^2/(2 mu_hl) Laplacian - v0 f(|xi|/sigma)] psi = E psi.  Sec. 5.1 fixes
the binding energy E = -E0 (E0 > 0) and solves the generalized eigenvalue
problem for the smallest depth v0:

    (T + E0) psi = v0 F psi,   T = -hbar^2/(2 mu_hl) D2,  F = diag f >= 0.

T + E0 is symmetric positive definite, so the v0 are the reciprocals of the
eigenvalues of the definite pencil (F, T + E0); the smallest positive v0 is
1 / lambda_max.  Solved with LAPACK (scipy.linalg.eigh, generalized form).
The grid is the periodic Fourier grid of ``grid`` (1D: n points on
[-L, L); 2D: the n x n tensor grid).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sl

from .grid import grid_points, d2_closed_form
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


def tune_v0(E0: float, mu_hl: float, sigma: float, shape: int, n: int, L: float,
            dim: int = 1, hbar: float = 1.0) -> float:
    """Smallest well depth v0 whose two-body ground state has energy -E0."""
    if not E0 > 0:
        raise ValueError("E0 must be positive")
    T, f = _kinetic_and_shape(dim, mu_hl, hbar, sigma, shape, n, L)
    A = T + E0 * np.eye(T.shape[0])
    lam = sl.eigh(np.diag(f), A, eigvals_only=True)
    return 1.0 / float(lam.max())


def two_body_energy(v0: float, mu_hl: float, sigma: float, shape: int, n: int, L: float,
                    dim: int = 1, hbar: float = 1.0) -> float:
    """Lowest eigenvalue of T - v0 F on the same grid."""
    T, f = _kinetic_and_shape(dim, mu_hl, hbar, sigma, shape, n, L)
    return float(np.linalg.eigvalsh(T - v0 * np.diag(f))[0])


def tune_v0_2d_iterative(E0: float, mu_hl: float, sigma: float, shape: int, n: int, L: float,
                         hbar: float = 1.0) -> float:
    """2D depth for grids too large for the dense pencil: the largest eigenvalue of the
    symmetric operator F^1/2 (T + E0)^-1 F^1/2 by ARPACK, with (T + E0)^-1 applied through
    LAPACK eigendecompositions of the 1D factors of T = -hbar^2/(2 mu) (D2 (x) I + I (x) D2)."""
    import scipy.sparse.linalg as spla
    if not E0 > 0:
        raise ValueError("E0 must be positive")
    x = grid_points(n, L)
    lam, S = np.linalg.eigh(-(hbar ** 2) / (2.0 * mu_hl) * d2_closed_form(n, L))
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
