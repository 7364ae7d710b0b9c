"""Shifted kinetic preconditioner (oracle; test infrastructure).

Sec. 4.2: the preconditioner neglects V and solves (T - theta) w = r with T
the kinetic Kronecker sum.  In 1D the paper writes this as the Sylvester
equation (Eq. sylvester_equation)

    (C1 - s1 I) W + W (C2 - s2 I)^T = B,   s1 + s2 = theta,

with W = reshape(w, N_y, N_x) (column-major, so W = P^T for P[i_x, j_y]),
C1 = a_y D2_y acting on y and C2 = a_x D2_x acting on x, and solves it with
Bartels-Stewart.  ``apply_sylvester`` does exactly that through
scipy.linalg.solve_sylvester (LAPACK Bartels-Stewart), splitting the shift
as the paper does, s_{1,2} proportional to the coefficients of y and x.
``apply_dense`` is the plain definition: a dense LU solve with the
assembled kinetic matrix.  ``kinetic_residual`` checks a candidate w at any
size through the explicit Kronecker apply.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sl

from .hamiltonian import Problem


def apply_dense(problem: Problem, r: np.ndarray, theta: float) -> np.ndarray:
    """(T - theta)^-1 r by a dense solve (small N only); r has shape [..., N]."""
    T = problem.kinetic_dense() - theta * np.eye(problem.N)
    r2 = np.asarray(r, dtype=np.float64).reshape(-1, problem.N)
    w = np.linalg.solve(T, r2.T).T
    return w.reshape(np.shape(r))


def apply_sylvester(problem: Problem, r: np.ndarray, theta: float) -> np.ndarray:
    """1D only: (T - theta)^-1 r through the Sylvester equation, one vector at a time."""
    if problem.dim != 1:
        raise ValueError("the Sylvester form is the 1D preconditioner")
    ax, ay = problem.a
    nx, ny = problem.n
    s1 = theta * ay / (ax + ay)
    s2 = theta * ax / (ax + ay)
    C1 = ay * problem.D2[1] - s1 * np.eye(ny)
    C2 = ax * problem.D2[0] - s2 * np.eye(nx)
    r2 = np.asarray(r, dtype=np.float64).reshape(-1, nx, ny)
    out = np.empty_like(r2)
    for b in range(r2.shape[0]):
        B = r2[b].T                                   # W layout: N_y x N_x
        W = sl.solve_sylvester(C1, C2.T, B)
        out[b] = W.T
    return out.reshape(np.shape(r))


def kinetic_residual(problem: Problem, w: np.ndarray, r: np.ndarray, theta: float) -> float:
    """max over vectors of ||(T - theta) w - r|| / ||r|| using the explicit Kronecker apply."""
    zero_v = Problem(problem.a, problem.n, problem.L, np.zeros(problem.n))
    w2 = np.asarray(w, dtype=np.float64).reshape(-1, problem.N)
    r2 = np.asarray(r, dtype=np.float64).reshape(-1, problem.N)
    res = zero_v.apply_kron(w2, theta) - r2
    return float(np.max(np.linalg.norm(res, axis=1) / np.linalg.norm(r2, axis=1)))
