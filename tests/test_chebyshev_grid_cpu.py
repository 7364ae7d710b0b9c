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
