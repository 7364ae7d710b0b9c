"""The library's host-side construction of the paper's mapped Chebyshev grid
(tps_chebyshev_grid, C++) against the oracle's (oracle/chebyshev.py, NumPy): the two are
written independently (the library takes the closed-form diagonal of the derivative
matrix, the oracle the negative row sum)."""
import numpy as np
import pytest

from oracle import chebyshev as cb


@pytest.mark.parametrize("n,L", [(2, 1.0), (8, 1.0), (33, 2.5), (64, 5.0), (128, 3.0)])
def test_chebyshev_grid_matches_oracle(n, L):
    from paper_2111_02534_gb300 import tps
    y, D2 = tps.chebyshev_grid(n, L)
    # the oracle forms y through sqrt(1 - t^2), which loses a few digits at the outer nodes
    assert np.max(np.abs(y - cb.mapped_points(n, L))) <= 1e-12 * np.abs(y).max()
    assert np.max(np.abs(D2 - cb.d2_mapped(n, L))) <= 1e-13 * np.abs(D2).max()


@pytest.mark.parametrize("n,L", [(1, 1.0), (1025, 1.0), (16, 0.0), (16, -2.0)])
def test_chebyshev_grid_rejects_bad_arguments(n, L):
    from paper_2111_02534_gb300 import tps
    with pytest.raises(tps.TpsError):
        tps.chebyshev_grid(n, L)


@pytest.mark.parametrize("n,L", [(2, 1.0), (16, 1.5), (64, 5.0), (128, 3.0)])
def test_fast_diagonalisation_factors(n, L):
    # the library's host QR eigensolver: D2 = S diag(lam) S^-1 with the oracle's (LAPACK)
    # eigenvalues, unit columns, S S^-1 = I
    from paper_2111_02534_gb300 import tps
    y, D2, lam, S, Sinv = tps.chebyshev_grid(n, L, factors=True)
    nrm = np.abs(D2).max()
    assert np.max(np.abs(lam - cb.lowest_eigenvalues(cb.d2_mapped(n, L), n))) <= 1e-13 * nrm
    assert np.all(np.diff(lam) >= 0)
    assert np.max(np.abs(D2 @ S - S * lam)) <= 1e-13 * nrm
    assert np.max(np.abs(np.linalg.norm(S, axis=0) - 1.0)) <= 1e-14
    assert np.max(np.abs(S @ Sinv - np.eye(n))) <= 1e-12


def test_preconditioner_from_library_factors_matches_oracle():
    # the Sec. 4.2 kinetic solve on the mapped grid built from the library's factors equals
    # the oracle's Bartels-Stewart solution
    from paper_2111_02534_gb300 import tps
    from oracle.hamiltonian import coefficients_from_alpha
    ax, ay = coefficients_from_alpha(20.0)
    n, L, theta = (24, 16), (1.5, 4.0), -0.4
    _, _, lx, Sx, Six = tps.chebyshev_grid(n[0], L[0], factors=True)
    _, _, ly, Sy, Siy = tps.chebyshev_grid(n[1], L[1], factors=True)
    R = np.random.default_rng(2).standard_normal(n)
    X = Sx @ ((Six @ R @ Siy.T) / (ax * lx[:, None] + ay * ly[None, :] - theta)) @ Sy.T
    ref = cb.kinetic_sylvester_solve((ax, ay), n, L, theta, R)
    assert np.max(np.abs(X - ref)) <= 1e-12 * np.abs(ref).max()
