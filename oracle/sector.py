"""Heavy-exchange parity sectors (oracle; test infrastructure).

Exchanging the two heavy particles flips the heavy-heavy Jacobi vector,
x -> -x (1D) or (x1, x2) -> (-x1, -x2) (2D), and leaves y unchanged.  The
potential of Eq. definition_potential is invariant under it, so H splits
into an even (bosonic) and an odd (fermionic) block -- the parity selection
rule of Sec. 5.1.  On the grid x_j = -L + j 2L/n the reflection is the
index permutation j -> (n - j) mod n.

The sector basis is built from its definition for any involutive
permutation R of the x indices: for each orbit {p, R p} with p != R p the
vector (e_p +/- e_{Rp}) / sqrt(2), and for each fixed point e_p (even only).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .grid import reflection_index

ANY = 0
X_EVEN = 1
X_ODD = 2


def involution_basis(perm: np.ndarray, sign: int) -> np.ndarray:
    """Orthonormal basis (columns) of {v : v[perm] = sign * v}."""
    n = perm.size
    cols = []
    for p in range(n):
        q = int(perm[p])
        if q == p:
            if sign > 0:
                e = np.zeros(n)
                e[p] = 1.0
                cols.append(e)
        elif p < q:
            e = np.zeros(n)
            e[p] = 1.0 / np.sqrt(2.0)
            e[q] = sign / np.sqrt(2.0)
            cols.append(e)
    return np.stack(cols, axis=1)


def x_reflection_perm(n_x) -> np.ndarray:
    """Permutation of the combined x index for x -> -x (1D: n_x int; 2D: (n_x1, n_x2))."""
    if np.isscalar(n_x):
        return reflection_index(int(n_x))
    n1, n2 = n_x
    r1, r2 = reflection_index(n1), reflection_index(n2)
    i1, i2 = np.meshgrid(np.arange(n1), np.arange(n2), indexing="ij")
    return (r1[i1] * n2 + r2[i2]).ravel()


def sector_basis(problem, parity: int):
    """Sparse N x N_s matrix B whose columns span the chosen sector (x-part (x) I_y)."""
    d = problem.dim
    n_x = problem.n[:d]
    n_y_total = int(np.prod(problem.n[d:]))
    if parity == ANY:
        return sp.identity(problem.N, format="csr")
    perm = x_reflection_perm(n_x[0] if d == 1 else n_x)
    Bx = involution_basis(perm, +1 if parity == X_EVEN else -1)
    return sp.kron(sp.csr_matrix(Bx), sp.identity(n_y_total), format="csr")


def reflect_x(problem, psi: np.ndarray) -> np.ndarray:
    """R_x psi for psi of shape [..., N]."""
    d = problem.dim
    perm = x_reflection_perm(problem.n[0] if d == 1 else problem.n[:d])
    n_y_total = int(np.prod(problem.n[d:]))
    lead = psi.shape[:-1]
    P = psi.reshape(lead + (perm.size, n_y_total))
    return P[..., perm, :].reshape(psi.shape)
