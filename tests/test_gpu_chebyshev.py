"""The paper's own discretisation on the GPU (Sec. 3.1: Chebyshev roots mapped to the real
line, dense non-symmetric D2; Sec. 4.1: Jacobi-Davidson for the non-symmetric H; Sec. 4.2:
fast diagonalisation with S^-1): the H-apply against the oracle's dense matrix, the
preconditioner against the oracle's Sylvester solve, and Table 1's lowest boson and fermion
at E0 = 0.1 (alpha = 20) on a 64 x 64 grid, against the oracle's dense eigenvalues and the
paper's printed values."""
import json
import os

import numpy as np
import pytest

from gpu_common import torch, require_gpu, dev, host
from oracle import chebyshev as cb
from oracle.hamiltonian import coefficients_from_alpha, GAUSS
from paper_2111_02534_gb300.inputs import random_block

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _ctx(n, L, v0, alpha=20.0):
    from paper_2111_02534_gb300 import tps
    ctx = tps.Context(1, 0)
    ctx.set_alpha(alpha)
    ctx.set_grid_chebyshev(list(n), list(L))
    ctx.set_pair_potential(tps.GAUSS, v0, 1.0)
    return ctx


@pytest.mark.parametrize("n,L", [((12, 10), (1.5, 3.0)), ((64, 64), (1.5, 5.0))])
def test_apply_h_and_prec_chebyshev(n, L):
    require_gpu()
    from paper_2111_02534_gb300 import tps
    ax, ay = coefficients_from_alpha(20.0)
    v0 = 0.3
    ctx = _ctx(n, L, v0)
    H = cb.hamiltonian_1d((ax, ay), n, L, v0, 1.0, GAUSS)
    psi = random_block(3, n[0] * n[1], 4)
    out = torch.empty(3, n[0] * n[1], dtype=torch.float64, device="cuda")
    scale = np.abs(H).max() * np.abs(psi).max() * max(n)
    for dt in (tps.F64, tps.F64_TC):
        ctx.apply_h(dev(psi), out, -0.2, dtype=dt)
        ctx.device_status()
        ref = psi @ (H - (-0.2) * np.eye(H.shape[0])).T
        assert np.max(np.abs(host(out) - ref)) <= 1e-13 * scale
    theta = -0.7
    ctx.apply_prec(dev(psi), out, theta, dtype=tps.F64)
    for v in range(3):
        ref = cb.kinetic_sylvester_solve((ax, ay), n, L, theta, psi[v])
        assert np.max(np.abs(host(out)[v] - ref.ravel())) <= 1e-9 * np.abs(ref).max()
    ctx.close()


@pytest.mark.parametrize("parity,key,nk", [(1, "bosons", 2), (2, "fermions", 1)])
def test_table1_on_the_gpu(parity, key, nk):
    """E0 = 0.1, alpha = 20, 64 x 64 mapped grid (map parameters 1.5 in x, 5 in y), v0 from
    the two-body problem on the mapped grid: the lowest bosons (x-even) and fermion (x-odd)
    of Table 1; against the oracle's dense eigenvalues of the same matrix to 1e-10 and the
    paper's printed ratios E/E0 (the ground states to half a unit of the 8th decimal, the
    first excited boson to the 7th, as the oracle itself reaches on this grid)."""
    require_gpu()
    from paper_2111_02534_gb300 import tps
    with open(os.path.join(GOLD, "table1.json")) as f:
        row = json.load(f)["rows"][0]
    ax, ay = coefficients_from_alpha(20.0)
    v0 = cb.tune_v0(row["E0"], 1.0, 1.0, GAUSS, 96, 4.0)
    n, L = (64, 64), (1.5, 5.0)
    ctx = _ctx(n, L, v0)
    ev = torch.empty(nk, n[0] * n[1], dtype=torch.float64, device="cuda")
    opts = tps.default_opts()
    lam, st = ctx.solve(nk, parity, 1e-12, 4, ev, opts=opts)
    H = cb.hamiltonian_1d((ax, ay), n, L, v0, 1.0, GAUSS)
    B = cb.x_sector_basis(n[0], n[1], +1 if parity == 1 else -1)
    ref = cb.lowest_eigenvalues(B.T @ H @ B, nk)
    assert np.max(np.abs(lam - ref) / np.abs(ref)) <= 1e-10, (lam, ref)
    ratios = np.asarray(lam) / row["E0"]
    assert abs(ratios[0] - row[key][0]) <= 5e-9
    if nk > 1:
        assert abs(ratios[1] - row[key][1]) <= 1e-7
    # the returned vectors are eigenvectors of the full-grid H with the sector's parity
    X = host(ev)
    for i in range(nk):
        r = H @ X[i] - lam[i] * X[i]
        assert np.linalg.norm(r) <= 1e-9 * np.abs(H).max()
        Xm = X[i].reshape(n)[::-1]
        assert np.allclose(Xm.ravel(), (1 if parity == 1 else -1) * X[i], atol=1e-12)
    ctx.close()
