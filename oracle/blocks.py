"""Block linear-algebra definitions behind the Jacobi-Davidson steps (oracle; test infrastructure).

Sec. 4.1: JDQR expands an orthonormal search space Q, takes Ritz pairs from
it, and solves the projected correction equation (Eq. jdcor)

    (I - Qt Qt^T)(A - theta I)(I - Qt Qt^T) dq = -(A q - q theta),  dq _|_ Qt,

with GMRES, preconditioned (Sec. 4.2).  For a symmetric A the Newton
system of Eq. jdqr reduces to Ritz pairs of Q^T A Q.  These are the plain
definitions the GPU building blocks are compared against; each is a few
lines of NumPy on top of LAPACK.
"""
from __future__ import annotations

import numpy as np


def gram(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A^T B for column blocks A [N, p], B [N, q]."""
    return A.T @ B


def rayleigh_ritz(V: np.ndarray, HV: np.ndarray):
    """Ritz values/vectors of the search space V (orthonormal columns, [N, m]).

    Returns theta (ascending), Y, X = V Y, R = HV Y - X diag(theta)."""
    G = V.T @ HV
    G = 0.5 * (G + G.T)
    theta, Y = np.linalg.eigh(G)
    X = V @ Y
    R = HV @ Y - X * theta[None, :]
    return theta, Y, X, R


def orthonormal_complement_step(Q: np.ndarray, T: np.ndarray) -> np.ndarray:
    """The definition of expanding an orthonormal basis Q [N, m] by a block T [N, b]:
    an orthonormal basis of span(Q, T) minus span(Q), via Householder QR of [Q, T]."""
    Z, _ = np.linalg.qr(np.concatenate([Q, T], axis=1))
    return Z[:, Q.shape[1]:]


def project_out(Q: np.ndarray, x: np.ndarray) -> np.ndarray:
    """(I - Q Q^T) x."""
    return x - Q @ (Q.T @ x)


def projected_preconditioner(Kinv, Qt: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Ktilde^-1 y = K^-1 y - K^-1 Qt (Qt^T K^-1 Qt)^-1 Qt^T K^-1 y: the inverse of
    (I - Qt Qt^T) K (I - Qt Qt^T) on the complement of Qt (Sleijpen-van der Vorst form)."""
    KQ = Kinv(Qt)
    M = Qt.T @ KQ
    z = Kinv(y)
    return z - KQ @ np.linalg.solve(M, Qt.T @ z)


def correction_exact(H: np.ndarray, Qt: np.ndarray, theta: float, r: np.ndarray) -> np.ndarray:
    """The exact solution dq _|_ Qt of Eq. jdcor for a dense symmetric H (small N only)."""
    N = H.shape[0]
    # orthonormal basis of the complement of Qt
    Z, _ = np.linalg.qr(np.concatenate([Qt, np.eye(N)], axis=1))
    C = Z[:, Qt.shape[1]:N]
    A = C.T @ (H - theta * np.eye(N)) @ C
    return C @ np.linalg.solve(A, -(C.T @ r))


def gmres(apply_A, b: np.ndarray, steps: int):
    """Textbook GMRES from x0 = 0: Arnoldi (modified Gram-Schmidt) for ``steps`` steps,
    then the least-squares problem min ||beta e1 - Hbar y|| by LAPACK.
    Returns (x, residual norm of the small problem after each step)."""
    n = b.size
    beta = np.linalg.norm(b)
    Vk = np.zeros((n, steps + 1))
    Hb = np.zeros((steps + 1, steps))
    Vk[:, 0] = b / beta
    res = []
    m = steps
    for j in range(steps):
        w = apply_A(Vk[:, j])
        for i in range(j + 1):
            Hb[i, j] = Vk[:, i] @ w
            w = w - Hb[i, j] * Vk[:, i]
        Hb[j + 1, j] = np.linalg.norm(w)
        e1 = np.zeros(j + 2)
        e1[0] = beta
        y, *_ = np.linalg.lstsq(Hb[:j + 2, :j + 1], e1, rcond=None)
        res.append(float(np.linalg.norm(e1 - Hb[:j + 2, :j + 1] @ y)))
        if Hb[j + 1, j] == 0.0:
            m = j + 1
            break
        Vk[:, j + 1] = w / Hb[j + 1, j]
    e1 = np.zeros(m + 1)
    e1[0] = beta
    y, *_ = np.linalg.lstsq(Hb[:m + 1, :m], e1, rcond=None)
    return Vk[:, :m] @ y, res
