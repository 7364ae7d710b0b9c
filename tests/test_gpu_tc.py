"""GPU parity of the tensor-core FP64 H-apply (TPS_F64_TC: Eq. tensor_op1D with the mode
products emulated on tcgen05 by error-free BF16 digit splitting) against the oracle and
against the FP64-FMA path, and of the solver when its FP64 H-applies use it.

Tolerances: the same as the FP64 path against the oracle (1e-12 of ||H||_est ||psi||
norm-wise, 1e-12 of ||H||_est max|psi| per element).  Against the FP64-FMA path on the
same input: 1e-14 of ||H||_est ||psi|| norm-wise -- both are within a few units of
2^-53 n of the row-max x column-max scale of every product (the splitting keeps 54 bits
of every operand row and drops only digit pairs below 2^-60 of it).
"""
import json
import os

import numpy as np
import pytest

from gpu_common import torch, require_gpu, make_ctx_1d, make_ctx_2d, dev, host
from oracle.hamiltonian import problem_1d
from oracle.eig import lowest_dense
from oracle.sector import X_EVEN as O_EVEN
from paper_2111_02534_gb300.inputs import random_block, random_normal_block, WORKLOADS

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _tps():
    from paper_2111_02534_gb300 import tps
    return tps


@pytest.mark.parametrize("n,nvec,theta", [((64, 64), 4, 0.0), ((100, 70), 3, -0.37),
                                          ((12, 8), 5, 0.5), ((130, 200), 2, 1.25),
                                          ((4, 4), 1, 0.0), ((258, 136), 2, 0.0)])
def test_apply_h_tc_vs_oracle(n, nvec, theta):
    require_gpu()
    tps = _tps()
    P = problem_1d(20.0, 1.0, 1.0, n, (20.0, 15.0), 1.0, 1.0)
    ctx = make_ctx_1d(20.0, 1.0, n, (20.0, 15.0), 1.0, 1.0)
    psi = random_block(nvec, P.N, 7 + nvec)
    out = torch.empty(nvec, P.N, dtype=torch.float64, device="cuda")
    ctx.apply_h(dev(psi), out, theta, dtype=tps.F64_TC)
    ctx.device_status()
    got = host(out)
    ref = P.apply_kron(psi, theta)
    hn = P.norm_estimate()
    err = np.linalg.norm(got - ref, axis=1) / (hn * np.linalg.norm(psi, axis=1))
    assert err.max() <= 1e-12, err.max()
    assert np.max(np.abs(got - ref)) <= 1e-12 * hn * np.abs(psi).max()
    ctx.close()


@pytest.mark.parametrize("n,nvec", [((512, 512), 30), ((258, 512), 9), ((384, 384), 4)])
def test_apply_h_tc_matches_fp64_path(n, nvec):
    # full-size grids, ragged tiles (258 rows), more vectors than one slice workspace holds
    # (30 at n = 512); random and smooth inputs
    require_gpu()
    tps = _tps()
    ctx = make_ctx_1d(40.0, 1.0, n, (20.0, 20.0), 0.0185, 1.0)
    N, hn = ctx.info()
    psi = dev(random_normal_block(nvec, N, 3))
    x = np.linspace(-20, 20, n[0], endpoint=False)[:, None]
    y = np.linspace(-20, 20, n[1], endpoint=False)[None, :]
    psi[0] = dev(np.exp(-0.05 * x * x - 0.3 * y * y).ravel())
    a = torch.empty_like(psi)
    b = torch.empty_like(psi)
    ctx.apply_h(psi, a, 0.0, dtype=tps.F64)
    ctx.apply_h(psi, b, 0.0, dtype=tps.F64_TC)
    ctx.device_status()
    d = (a - b).norm(dim=1) / (hn * psi.norm(dim=1))
    assert float(d.max()) <= 1e-14, float(d.max())
    # the same answer on a second call (slices rebuilt in the reused workspace)
    c = torch.empty_like(psi)
    ctx.apply_h(psi, c, 0.0, dtype=tps.F64_TC)
    torch.cuda.synchronize()
    assert torch.equal(b, c)
    ctx.close()


def test_apply_h_tc_full_size_vs_oracle():
    """The 512 x 512 grid with 30 vectors (more than one slice-workspace chunk of 27):
    sampled rows of the first and last vectors against the oracle's row-by-row apply."""
    require_gpu()
    tps = _tps()
    P = problem_1d(40.0, 1.0, 1.0, (512, 512), (20.0, 20.0), 0.0185, 1.0)
    ctx = make_ctx_1d(40.0, 1.0, (512, 512), (20.0, 20.0), 0.0185, 1.0)
    N, hn = ctx.info()
    nvec = 30
    psi = random_normal_block(nvec, N, 13)
    out = torch.empty(nvec, N, dtype=torch.float64, device="cuda")
    ctx.apply_h(dev(psi), out, -0.01, dtype=tps.F64_TC)
    ctx.device_status()
    got = host(out)
    rows = np.random.default_rng(17).choice(N, 96, replace=False)
    for v in (0, 26, 27, nvec - 1):
        ref = P.apply_rows(psi[v], rows, -0.01)
        assert np.max(np.abs(got[v][rows] - ref)) <= 1e-12 * hn * np.abs(psi[v]).max()
    ctx.close()


@pytest.mark.parametrize("n,nvec,theta", [((8, 8, 6, 6), 2, 0.0), ((6, 6, 10, 10), 3, -0.4),
                                          ((12, 12, 8, 8), 1, 0.7), ((4, 4, 4, 4), 2, 0.0),
                                          ((128, 128, 4, 4), 2, 0.3),
                                          ((4, 4, 128, 128), 1, -0.2)])
def test_apply_h_tc_2d_vs_oracle(n, nvec, theta):
    """Eq. tensor_op2D with the four mode products on the tensor cores, against the
    oracle's Kronecker-sum apply, element by element (the same bar as the FP64 path).  The
    128-point modes are the longest contraction the 2D digit format takes (base-256 digits,
    level sums exact up to 146 points), as fibers of stride > 1 and as rows."""
    require_gpu()
    tps = _tps()
    from oracle.hamiltonian import problem_2d
    L = (5.0, 5.0, 4.0, 4.0)
    P = problem_2d(20.0, 1.0, 1.0, n, L, 2.0, 1.0)
    ctx = make_ctx_2d(20.0, 1.0, n, L, 2.0, 1.0)
    psi = random_block(nvec, P.N, 11 + nvec)
    out = torch.empty(nvec, P.N, dtype=torch.float64, device="cuda")
    ctx.apply_h(dev(psi), out, theta, dtype=tps.F64_TC)
    ctx.device_status()
    got = host(out)
    ref = P.apply_kron(psi, theta)
    hn = P.norm_estimate()
    err = np.linalg.norm(got - ref, axis=1) / (hn * np.linalg.norm(psi, axis=1))
    assert err.max() <= 1e-12, err.max()
    assert np.max(np.abs(got - ref)) <= 1e-12 * hn * np.abs(psi).max()
    ctx.close()


def test_apply_h_tc_2d_full_size():
    """The 48^4 workload (5.3 M unknowns) with more vectors than one fiber-slice chunk:
    sampled rows against the oracle, whole vectors against the FP64-FMA path, and the same
    bits on a second call."""
    require_gpu()
    tps = _tps()
    from oracle.hamiltonian import problem_2d
    w = WORKLOADS["2d_n48"]
    P = problem_2d(w.M, w.m, w.hbar, w.n, w.L, w.v0, w.sigma)
    ctx = make_ctx_2d(w.M, w.m, w.n, w.L, w.v0, w.sigma)
    N, hn = ctx.info()
    nvec = 12
    psi = dev(random_normal_block(nvec, N, 5))
    a = torch.empty_like(psi)
    b = torch.empty_like(psi)
    ctx.apply_h(psi, a, -0.3, dtype=tps.F64)
    ctx.apply_h(psi, b, -0.3, dtype=tps.F64_TC)
    ctx.device_status()
    d = (a - b).norm(dim=1) / (hn * psi.norm(dim=1))
    assert float(d.max()) <= 1e-14, float(d.max())
    rows = np.random.default_rng(3).choice(N, 48, replace=False)
    ph = host(psi)
    got = host(b)
    for v in (0, nvec - 1):
        ref = P.apply_rows(ph[v], rows, -0.3)
        assert np.max(np.abs(got[v][rows] - ref)) <= 1e-12 * hn * np.abs(ph[v]).max()
    c = torch.empty_like(psi)
    ctx.apply_h(psi, c, -0.3, dtype=tps.F64_TC)
    torch.cuda.synchronize()
    assert torch.equal(b, c)
    ctx.close()


@pytest.mark.parametrize("h_dtype", [0, 1])
def test_solve_with_tc_products_small(h_dtype):
    require_gpu()
    tps = _tps()
    w = WORKLOADS["1d_n64"]
    P = problem_1d(w.M, w.m, w.hbar, w.n, w.L, w.v0, w.sigma)
    ctx = make_ctx_1d(w.M, w.m, w.n, w.L, w.v0, w.sigma)
    ev = torch.empty(w.k, P.N, dtype=torch.float64, device="cuda")
    opts = tps.default_opts()
    opts.h_dtype = h_dtype
    opts.h64_dtype = tps.F64_TC
    lam, st = ctx.solve(w.k, tps.X_EVEN, 1e-12, w.block, ev, opts=opts)
    ref, _ = lowest_dense(P, w.k, O_EVEN)
    assert np.max(np.abs(lam - ref) / np.abs(ref)) <= 1e-10
    ctx.close()


def test_solve_with_tc_products_full_size():
    require_gpu()
    tps = _tps()
    w = WORKLOADS["1d_n512"]
    with open(os.path.join(GOLD, "evals_1d_n512.json")) as f:
        gold = json.load(f)
    ctx = make_ctx_1d(w.M, w.m, w.n, w.L, gold["v0"], w.sigma)
    ev = torch.empty(w.k, ctx.info()[0], dtype=torch.float64, device="cuda")
    opts = tps.default_opts()
    opts.h64_dtype = tps.F64_TC
    lam, st = ctx.solve(w.k, tps.X_EVEN, 1e-12, w.block, ev, opts=opts)
    ref = np.array(gold["evals"])
    assert np.max(np.abs(lam - ref) / np.maximum(np.abs(ref), abs(ref[0]))) <= 1e-10
    ctx.close()


def test_bounded_wait_reports_timeout_and_the_device_stays_usable():
    # the tensor-core kernels' waits give up after a bounded time and report it instead
    # of hanging; the self-test takes that path on purpose (a barrier nothing signals)
    require_gpu()
    tps = _tps()
    assert tps._lib.tps_selftest_wait_timeout(0, 0.2) == tps.ERR_TIMEOUT
    assert tps._lib.tps_selftest_wait_timeout(0, 0.0) == tps.ERR_INVALID_ARG
    # afterwards the library's kernels run and agree as before
    ctx = make_ctx_1d(20.0, 1.0, (64, 64), (20.0, 20.0), 1.0, 1.0)
    N, hn = ctx.info()
    psi = dev(random_normal_block(2, N, 4))
    a, b = torch.empty_like(psi), torch.empty_like(psi)
    ctx.apply_h(psi, a, 0.0, dtype=tps.F64)
    ctx.apply_h(psi, b, 0.0, dtype=tps.F64_TC)
    ctx.device_status()
    assert float(((a - b).norm(dim=1) / (hn * psi.norm(dim=1))).max()) <= 1e-14
    ctx.close()
