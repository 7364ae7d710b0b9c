"""The paper's own discretisation: collocation on the roots of a Chebyshev polynomial, mapped
to the real line by an algebraic map (oracle; test infrastructure).

Sec. 3.1 names the basis (Chebyshev polynomials on a finite interval), the grid (their
roots) and an algebraic map to the infinite line (Boyd), and states that the resulting
second-derivative matrices are dense and in general non-symmetric; it prints no formulas.
Written out here (the reading is recorded with the others):

* nodes: the roots of T_n, t_j = -cos(pi (j + 1/2) / n), j = 0 .. n-1 (ascending);
* barycentric weights of these nodes (Berrut & Trefethen, SIAM Review 46, 2004), in closed
  form w_j = (-1)^j sin(pi (j + 1/2) / n) up to a common factor (the tests pin this to the
  product definition 1 / prod_{k != j} (t_j - t_k));
* first-derivative collocation matrix of the interpolating polynomial:
  D_ij = (w_j / w_i) / (t_i - t_j) for i != j, D_ii = -sum_{j != i} D_ij;
* the algebraic map y = L t / sqrt(1 - t^2) (t = y / sqrt(L^2 + y^2)), so that
  dt/dy = (1 - t^2)^(3/2) / L and d^2t/dy^2 = -3 t (1 - t^2)^2 / L^2;
* second derivative in y by the chain rule:
  D2_y = diag((dt/dy)^2) D D + diag(d^2t/dy^2) D.

The three-body matrix is the same Kronecker sum as on the Fourier grid (Eq.
discretized_Schroedinger_equation_1D), H = a_x (D2_x (x) I) + a_y (I (x) D2_y) + diag(V),
now non-symmetric; its eigenvalues are computed by LAPACK's general solver.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sl

from .hamiltonian import pair_potential_1d, shape_function


def nodes(n: int) -> np.ndarray:
    """Roots of T_n on [-1, 1], ascending."""
    j = np.arange(n)
    return -np.cos(np.pi * (j + 0.5) / n)


def weights(n: int) -> np.ndarray:
    """Barycentric weights of ``nodes(n)`` (closed form, common factor dropped)."""
    j = np.arange(n)
    # nodes(n)[j] = cos(theta_j) with theta_j = pi - pi (j + 1/2) / n; sin(theta_j) > 0
    return (-1.0) ** j * np.sin(np.pi * (j + 0.5) / n)


def d1(n: int) -> np.ndarray:
    """First-derivative collocation matrix on ``nodes(n)`` (exact for degree < n)."""
    t, w = nodes(n), weights(n)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (w[j] / w[i]) / (t[i] - t[j])
        D[i, i] = -np.sum(D[i, :])
    return D


def mapped_points(n: int, L: float) -> np.ndarray:
    """Grid on the real line: y_j = L t_j / sqrt(1 - t_j^2)."""
    t = nodes(n)
    return L * t / np.sqrt(1.0 - t * t)


def d2_mapped(n: int, L: float) -> np.ndarray:
    """d^2/dy^2 on the mapped grid (dense, non-symmetric)."""
    t = nodes(n)
    D = d1(n)
    tp = (1.0 - t * t) ** 1.5 / L            # dt/dy
    tpp = -3.0 * t * (1.0 - t * t) ** 2 / L ** 2  # d^2t/dy^2
    return np.diag(tp * tp) @ (D @ D) + np.diag(tpp) @ D


def hamiltonian_1d(a, n, L, v0: float, sigma: float, shape: int) -> np.ndarray:
    """Dense three-body H on the mapped grids: a = (a_x, a_y), n = (n_x, n_y), L = (L_x,
    L_y); vector index i n_y + j (x slow)."""
    x, y = mapped_points(n[0], L[0]), mapped_points(n[1], L[1])
    V = pair_potential_1d(x, y, v0, sigma, shape)
    H = a[0] * np.kron(d2_mapped(n[0], L[0]), np.eye(n[1]))
    H += a[1] * np.kron(np.eye(n[0]), d2_mapped(n[1], L[1]))
    H += np.diag(V.ravel())
    return H


def x_sector_basis(nx: int, ny: int, parity: int) -> np.ndarray:
    """Orthonormal basis of the functions even (parity +1) or odd (-1) under x -> -x; the
    node set is symmetric (x_i -> x_{n-1-i}) and has no node at 0 for even n."""
    if nx % 2:
        raise ValueError("n_x must be even")
    cols = []
    for i in range(nx // 2):
        for j in range(ny):
            v = np.zeros((nx, ny))
            v[i, j] = 1.0 / np.sqrt(2.0)
            v[nx - 1 - i, j] = parity / np.sqrt(2.0)
            cols.append(v.ravel())
    return np.stack(cols, axis=1)


def lowest_eigenvalues(H: np.ndarray, k: int) -> np.ndarray:
    """The k smallest eigenvalues of a real non-symmetric matrix with a real spectrum
    (imaginary parts must be negligible)."""
    lam = sl.eigvals(H)
    if np.max(np.abs(lam.imag)) > 1e-8 * np.max(np.abs(lam)):
        raise ValueError("complex eigenvalues")
    return np.sort(lam.real)[:k]


def tune_v0(E0: float, mu_hl: float, sigma: float, shape: int, n: int, L: float,
            hbar: float = 1.0) -> float:
    """Smallest depth v0 with a two-body ground state at -E0 on the mapped grid: the
    generalized problem (T + E0) psi = v0 F psi (Sec. 5.1) as the largest eigenvalue mu of
    (T + E0)^-1 F, v0 = 1 / mu (F is nearly singular far out, T + E0 is not)."""
    if not E0 > 0:
        raise ValueError("E0 must be positive")
    y = mapped_points(n, L)
    T = -(hbar ** 2) / (2.0 * mu_hl) * d2_mapped(n, L)
    F = np.diag(shape_function(np.abs(y) / sigma, shape))
    mu = sl.eigvals(sl.solve(T + E0 * np.eye(n), F))
    return float(1.0 / np.max(mu.real))


def tune_v0_2d(E0: float, mu_hl: float, sigma: float, shape: int, n: int, L: float,
               hbar: float = 1.0) -> float:
    """The 2D two-body depth (Sec. 5.2) on the n x n tensor grid of mapped points: the same
    generalized problem with T = -hbar^2/(2 mu_hl) (D2 (x) I + I (x) D2) and
    F = diag f(|xi| / sigma), dense (n^2 unknowns)."""
    if not E0 > 0:
        raise ValueError("E0 must be positive")
    y = mapped_points(n, L)
    T1 = -(hbar ** 2) / (2.0 * mu_hl) * d2_mapped(n, L)
    I = np.eye(n)
    T = np.kron(T1, I) + np.kron(I, T1)
    Y1, Y2 = np.meshgrid(y, y, indexing="ij")
    F = np.diag(shape_function(np.sqrt(Y1 ** 2 + Y2 ** 2).ravel() / sigma, shape))
    mu = sl.eigvals(sl.solve(T + E0 * np.eye(n * n), F))
    return float(1.0 / np.max(mu.real))


def kinetic_sylvester_solve(a, n, L, theta: float, R: np.ndarray) -> np.ndarray:
    """The preconditioner of Sec. 4.2 on the mapped grid (V neglected): X with
    a_x D2_x X + a_y X D2_y^T - theta X = R (R, X: n_x x n_y, x slow), i.e.
    (a_x D2_x (x) I + a_y I (x) D2_y - theta) vec X = vec R, solved as a Sylvester equation
    by Bartels-Stewart (scipy.linalg.solve_sylvester), the paper's 1D method (Eq.
    sylvester_equation)."""
    A = a[0] * d2_mapped(n[0], L[0]) - theta * np.eye(n[0])
    B = (a[1] * d2_mapped(n[1], L[1])).T
    return sl.solve_sylvester(A, B, np.asarray(R, dtype=np.float64).reshape(n[0], n[1]))


def kinetic_fast_diag_solve(a, n, L, theta: float, R: np.ndarray) -> np.ndarray:
    """The same solve by fast diagonalisation, D2_k = S_k diag(lam_k) S_k^-1 (a real
    spectrum, non-orthogonal S_k): X = S_x [(S_x^-1 R S_y^-T) ./ (a_x lam_x + a_y lam_y -
    theta)] S_y^T."""
    lx, Sx = np.linalg.eig(d2_mapped(n[0], L[0]))
    ly, Sy = np.linalg.eig(d2_mapped(n[1], L[1]))
    if np.max(np.abs(lx.imag)) > 0 or np.max(np.abs(ly.imag)) > 0:
        raise ValueError("complex spectrum")
    lx, Sx, ly, Sy = lx.real, Sx.real, ly.real, Sy.real
    Rt = np.linalg.solve(Sx, np.asarray(R, dtype=np.float64).reshape(n[0], n[1]))
    Rt = np.linalg.solve(Sy, Rt.T).T
    Xt = Rt / (a[0] * lx[:, None] + a[1] * ly[None, :] - theta)
    return Sx @ Xt @ Sy.T
