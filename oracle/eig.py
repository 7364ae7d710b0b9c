"""Lowest eigenpairs of the discrete three-body Hamiltonian (oracle; test infrastructure).

The paper's eigensolvers (Krylov-Schur, JDQR; Sec. 4.1, Sec. 5.1) all
converge to the same thing: the lowest eigenpairs of the matrix H of Eq.
matrix_evp in a parity sector.  The oracle computes that thing directly:

* ``lowest_dense``     -- dense LAPACK eigh of B^T H B, H assembled
                          explicitly, B the sector basis (N_s up to ~10^4).
* ``lowest_iterative`` -- for larger grids, SciPy LOBPCG on B^T H B applied
                          through the Kronecker identity, preconditioned by
                          the inverse of the shifted kinetic part obtained
                          from LAPACK eigendecompositions of the dense D2
                          matrices.  The preconditioner only changes the
                          speed of convergence, never the limit.
* ``certify``          -- residual norms and the Weyl (|lambda - theta| <=
                          ||r||) and Kato-Temple (|lambda - theta| <=
                          ||r||^2 / gap) bounds for unit vectors.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .hamiltonian import Problem
from .sector import sector_basis


def lowest_dense(problem: Problem, k: int, parity: int):
    """(eigenvalues[k], eigenvectors[k, N]) of H in the sector, ascending."""
    B = sector_basis(problem, parity).toarray()
    H = problem.assemble_dense()
    Hs = B.T @ H @ B
    Hs = 0.5 * (Hs + Hs.T)
    w, Y = np.linalg.eigh(Hs)
    X = (B @ Y[:, :k]).T
    return w[:k], X


def all_eigenvalues_dense(problem: Problem, parity: int) -> np.ndarray:
    B = sector_basis(problem, parity).toarray()
    H = problem.assemble_dense()
    Hs = B.T @ H @ B
    return np.linalg.eigvalsh(0.5 * (Hs + Hs.T))


def lowest_iterative(problem: Problem, k: int, parity: int, tol: float = 1e-10,
                     extra: int = 4, seed: int = 0, maxiter: int = 2000, shift=None):
    """(eigenvalues[k], eigenvectors[k, N]) by LOBPCG in the sector.

    ``tol`` is the LOBPCG residual-norm tolerance relative to ||H||_est."""
    B = sector_basis(problem, parity)
    Ns = B.shape[1]
    N = problem.N
    hnorm = problem.norm_estimate()
    # kinetic eigendecompositions for the preconditioner (LAPACK, dense D2)
    lam, S = [], []
    for ak, D in zip(problem.a, problem.D2):
        w, U = np.linalg.eigh(ak * D)
        lam.append(w)
        S.append(U)
    den = lam[0]
    for l in lam[1:]:
        den = np.add.outer(den, l)
    sig = shift if shift is not None else min(float(problem.V.min()), -1e-3 * hnorm)

    def to_full(U):                      # [Ns, b] -> [b, N]
        return np.asarray(B @ U).T

    def to_sector(P):                    # [b, N] -> [Ns, b]
        return np.asarray(B.T @ P.T)

    def h_mat(U):
        U = U.reshape(Ns, -1)
        return to_sector(problem.apply_kron(to_full(U)))

    def p_mat(U):
        U = U.reshape(Ns, -1)
        P = to_full(U).reshape((-1,) + problem.n)
        T = P
        for m, Sm in enumerate(S):
            T = np.moveaxis(np.moveaxis(T, m + 1, -1) @ Sm, -1, m + 1)
        T = T / (den - sig)[None]
        for m, Sm in enumerate(S):
            T = np.moveaxis(np.moveaxis(T, m + 1, -1) @ Sm.T, -1, m + 1)
        return to_sector(T.reshape(-1, N))

    Hop = spla.LinearOperator((Ns, Ns), matvec=lambda v: h_mat(v).ravel(), matmat=h_mat,
                              dtype=np.float64)
    Pop = spla.LinearOperator((Ns, Ns), matvec=lambda v: p_mat(v).ravel(), matmat=p_mat,
                              dtype=np.float64)
    rng = np.random.default_rng(seed)
    X0 = rng.standard_normal((Ns, k + extra))
    w, U = spla.lobpcg(Hop, X0, M=Pop, tol=tol * hnorm, maxiter=maxiter, largest=False)
    order = np.argsort(w)
    w, U = w[order], U[:, order]
    # final Rayleigh-Ritz in FP64 with explicit normalisation
    Q, _ = np.linalg.qr(U)
    G = Q.T @ h_mat(Q)
    G = 0.5 * (G + G.T)
    th, Y = np.linalg.eigh(G)
    X = to_full(Q @ Y)
    return th[:k], X[:k]


def residual_norms(problem: Problem, X: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """||H x_i - theta_i x_i|| for unit-normalised rows x_i (explicit Kronecker apply)."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, problem.N)
    X = X / np.linalg.norm(X, axis=1, keepdims=True)
    HX = problem.apply_kron(X)
    return np.linalg.norm(HX - theta[:, None] * X, axis=1)


def rayleigh_quotients(problem: Problem, X: np.ndarray) -> np.ndarray:
    X = np.asarray(X, dtype=np.float64).reshape(-1, problem.N)
    HX = problem.apply_kron(X)
    return np.einsum("bi,bi->b", X, HX) / np.einsum("bi,bi->b", X, X)


def certify(theta: np.ndarray, resid: np.ndarray, spectrum: np.ndarray):
    """Weyl and Kato-Temple bounds on |lambda_i - theta_i| given a reference spectrum
    (the gap is the distance from theta_i to the nearest other reference eigenvalue)."""
    weyl = np.asarray(resid, dtype=np.float64)
    kt = np.empty_like(weyl)
    for i, t in enumerate(theta):
        d = np.abs(np.asarray(spectrum) - t)
        d_sorted = np.sort(d)
        gap = d_sorted[1] if d_sorted.size > 1 else np.inf
        kt[i] = weyl[i] ** 2 / gap if gap > weyl[i] else np.inf
    return weyl, kt
