"""Three-body Hamiltonian on the Fourier grid, assembled explicitly (oracle; test infrastructure).

Follows Sec. 2 and Sec. 3.1 of the paper:

* Eq. Schroedinger_equation_three_body: H = -(a_x-part) Laplacian_x -
  (a_y-part) Laplacian_y + V in Jacobi coordinates, written here as
  H = a_x * d^2/dx^2 + a_y * d^2/dy^2 + V with a_k = -hbar^2 / (2 mu_k).
  x is the heavy-heavy separation (reduced mass mu_x = M/2, the coefficient
  2/(1+alpha) of Sec. 2 in heavy-light units), y the light particle
  relative to the heavy pair's centre of mass (mu_y = 2Mm/(2M+m)).
* Eq. definition_potential: only heavy-light pairs interact,
  V = -v0 [f(|y - x/2| / sigma) + f(|y + x/2| / sigma)] (the light particle's
  distance to either heavy one), with f_G = exp(-xi^2) (Eq.
  Gaussian_shaped_potential) or f_L = (1 + xi^2)^-3 (Eq.
  Lorentzian_shaped_potential).  The potential is evaluated pointwise on
  the grid, not periodised.
* Eq. discretized_Schroedinger_equation_1D / Eq. Ham2D: the discrete H is the
  Kronecker sum a_x (D2_x (x) I_y) + a_y (I_x (x) D2_y) + diag(V), with the
  vector ordered psi_{i,j}, i the x index (slow), j the y index (fast)
  (Sec. 3.1).  In 2D the ordering is [x1][x2][y1][y2].

``assemble_dense`` / ``assemble_csr`` build the matrix literally with
Kronecker products.  ``apply_rows`` evaluates chosen rows of H psi one by one
from the same definition, for spot checks at sizes where assembly is too big.
``apply_kron`` applies the Kronecker sum through (A (x) B) vec(X) =
vec(A X B^T) (row-major vec); tests pin it to the explicit assembly.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .grid import grid_points, d2_closed_form

GAUSS = 0
LORENTZ3 = 1


def coefficients_from_masses(M: float, m: float, hbar: float = 1.0):
    """(a_x, a_y, mu_hl): a_k = -hbar^2/(2 mu_k), mu_x = M/2, mu_y = 2Mm/(2M+m), mu_hl = Mm/(M+m)."""
    mu_x = M / 2.0
    mu_y = 2.0 * M * m / (2.0 * M + m)
    mu_hl = M * m / (M + m)
    return -hbar ** 2 / (2.0 * mu_x), -hbar ** 2 / (2.0 * mu_y), mu_hl


def coefficients_from_alpha(alpha: float):
    """Paper units (heavy-light reduced mass 1, Sec. 2): a_x = -alpha_x/2, a_y = -alpha_y/2
    with alpha_x = 2/(1+alpha), alpha_y = (1+2 alpha)/(2+2 alpha)."""
    alpha_x = 2.0 / (1.0 + alpha)
    alpha_y = (1.0 + 2.0 * alpha) / (2.0 + 2.0 * alpha)
    return -alpha_x / 2.0, -alpha_y / 2.0


def shape_function(xi: np.ndarray, shape: int) -> np.ndarray:
    if shape == GAUSS:
        return np.exp(-xi * xi)
    if shape == LORENTZ3:
        return 1.0 / (1.0 + xi * xi) ** 3
    raise ValueError("unknown shape")


def pair_potential_1d(x: np.ndarray, y: np.ndarray, v0: float, sigma: float,
                      shape: int = GAUSS) -> np.ndarray:
    """V[i, j] = -v0 [f(|y_j - x_i/2|/sigma) + f(|y_j + x_i/2|/sigma)], shape [n_x, n_y]."""
    V = np.empty((x.size, y.size))
    for i in range(x.size):
        d_minus = np.abs(y - x[i] / 2.0) / sigma
        d_plus = np.abs(y + x[i] / 2.0) / sigma
        V[i, :] = -v0 * (shape_function(d_minus, shape) + shape_function(d_plus, shape))
    return V


def pair_potential_2d(x1, x2, y1, y2, v0: float, sigma: float, shape: int = GAUSS) -> np.ndarray:
    """V[i1,i2,j1,j2] = -v0 [f(|r_y - r_x/2|/sigma) + f(|r_y + r_x/2|/sigma)], r_x=(x1,x2), r_y=(y1,y2)."""
    X1, X2, Y1, Y2 = np.meshgrid(x1, x2, y1, y2, indexing="ij")
    d_minus = np.sqrt((Y1 - X1 / 2.0) ** 2 + (Y2 - X2 / 2.0) ** 2) / sigma
    d_plus = np.sqrt((Y1 + X1 / 2.0) ** 2 + (Y2 + X2 / 2.0) ** 2) / sigma
    return -v0 * (shape_function(d_minus, shape) + shape_function(d_plus, shape))


class Problem:
    """A discretised three-body problem: kinetic coefficients per coordinate,
    D2 per coordinate, potential V on the grid (C order = the vector ordering)."""

    def __init__(self, a, n, L, V):
        self.a = tuple(float(t) for t in a)          # one coefficient per coordinate
        self.n = tuple(int(t) for t in n)
        self.L = tuple(float(t) for t in L)
        self.V = np.asarray(V, dtype=np.float64).reshape(self.n)
        self.D2 = [d2_closed_form(nk, Lk) for nk, Lk in zip(self.n, self.L)]
        self.dim = len(self.n) // 2

    @property
    def N(self) -> int:
        return int(np.prod(self.n))

    def grids(self):
        return [grid_points(nk, Lk) for nk, Lk in zip(self.n, self.L)]

    def norm_estimate(self) -> float:
        """||H||_est = sum_k |a_k| (pi/h_k)^2 + max|V|  (h_k = 2 L_k / n_k)."""
        s = 0.0
        for ak, nk, Lk in zip(self.a, self.n, self.L):
            h = 2.0 * Lk / nk
            s += abs(ak) * (np.pi / h) ** 2
        return s + float(np.max(np.abs(self.V)))

    # ---- explicit assembly -------------------------------------------------
    def _mode_terms(self, sparse: bool):
        eye = (lambda k: sp.identity(k, format="csr")) if sparse else np.eye
        kron = (lambda A, B: sp.kron(A, B, format="csr")) if sparse else np.kron
        terms = []
        for k in range(len(self.n)):
            T = None
            for l in range(len(self.n)):
                F = (sp.csr_matrix(self.D2[l]) if sparse else self.D2[l]) if l == k else eye(self.n[l])
                T = F if T is None else kron(T, F)
            terms.append(self.a[k] * T)
        return terms

    def assemble_dense(self) -> np.ndarray:
        """H as a dense N x N matrix (small N only)."""
        H = np.diag(self.V.ravel()).astype(np.float64)
        for T in self._mode_terms(sparse=False):
            H = H + T
        return H

    def assemble_csr(self) -> sp.csr_matrix:
        """H as a SciPy CSR matrix built from Kronecker products."""
        H = sp.diags(self.V.ravel(), format="csr")
        for T in self._mode_terms(sparse=True):
            H = H + T
        return H.tocsr()

    def kinetic_dense(self) -> np.ndarray:
        """The kinetic part alone (V neglected), dense."""
        T = np.zeros((self.N, self.N))
        for t in self._mode_terms(sparse=False):
            T = T + t
        return T

    # ---- application without assembly --------------------------------------
    def apply_kron(self, psi: np.ndarray, theta: float = 0.0) -> np.ndarray:
        """(H - theta) psi for psi of shape [..., N] via (A (x) I) vec(X) = vec(A X) per mode."""
        psi = np.asarray(psi, dtype=np.float64)
        lead = psi.shape[:-1]
        P = psi.reshape((-1,) + self.n)
        out = (self.V[None] - theta) * P
        for k in range(len(self.n)):
            # contract mode k of P with a_k D2_k
            Pk = np.moveaxis(P, k + 1, -1)
            Rk = Pk @ (self.a[k] * self.D2[k]).T
            out = out + np.moveaxis(Rk, -1, k + 1)
        return out.reshape(lead + (self.N,))

    def apply_rows(self, psi: np.ndarray, rows: np.ndarray, theta: float = 0.0) -> np.ndarray:
        """((H - theta) psi)[r] for the flat indices r in ``rows``, each row computed on its
        own from the Kronecker-sum definition: row (i_1..i_d) of a_k (I (x) D2_k (x) I)
        holds a_k D2_k[i_k, i'] at the column that differs from r only in index k."""
        P = np.asarray(psi, dtype=np.float64).reshape(self.n)
        out = np.empty(len(rows))
        for t, r in enumerate(rows):
            idx = np.unravel_index(int(r), self.n)
            acc = (self.V[idx] - theta) * P[idx]
            for k in range(len(self.n)):
                line = list(idx)
                line[k] = slice(None)
                acc += self.a[k] * float(np.dot(self.D2[k][idx[k], :], P[tuple(line)]))
            out[t] = acc
        return out


def problem_1d(M, m, hbar, n, L, v0, sigma, shape=GAUSS, V=None, alpha=None) -> Problem:
    """1D problem from masses (or from alpha in heavy-light units when ``alpha`` is given)."""
    if alpha is not None:
        ax, ay = coefficients_from_alpha(alpha)
    else:
        ax, ay, _ = coefficients_from_masses(M, m, hbar)
    x = grid_points(n[0], L[0])
    y = grid_points(n[1], L[1])
    if V is None:
        V = pair_potential_1d(x, y, v0, sigma, shape)
    return Problem((ax, ay), n, L, V)


def problem_2d(M, m, hbar, n, L, v0, sigma, shape=GAUSS, V=None, alpha=None) -> Problem:
    """2D problem, ordering [x1][x2][y1][y2]."""
    if alpha is not None:
        ax, ay = coefficients_from_alpha(alpha)
    else:
        ax, ay, _ = coefficients_from_masses(M, m, hbar)
    g = [grid_points(nk, Lk) for nk, Lk in zip(n, L)]
    if V is None:
        V = pair_potential_2d(g[0], g[1], g[2], g[3], v0, sigma, shape)
    return Problem((ax, ax, ay, ay), n, L, V)
