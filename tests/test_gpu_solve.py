"""GPU parity of the block Jacobi-Davidson solver (Sec. 4.1, Sec. 4.2) against the oracle.

Bar: every returned eigenvalue within 1e-10 relative of the oracle's; eigenvectors
certified by the oracle's own residual ||H x - lambda x|| (Weyl / Kato-Temple bounds),
exchange parity exact, unit norm, sign convention.
"""
import json
import os

import numpy as np
import pytest

from gpu_common import torch, require_gpu, make_ctx_1d, make_ctx_2d, dev, host
from oracle.hamiltonian import problem_1d, problem_2d, Problem, coefficients_from_masses, GAUSS
from oracle.eig import lowest_dense, all_eigenvalues_dense, residual_norms, certify
from oracle.sector import reflect_x, ANY as O_ANY, X_EVEN as O_EVEN, X_ODD as O_ODD
from oracle.two_body import tune_v0
from paper_2111_02534_gb300.inputs import WORKLOADS

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _tps():
    from paper_2111_02534_gb300 import tps
    return tps


def _solve(ctx, k, parity, block, tol=1e-12, **kw):
    N = ctx.info()[0]
    ev = torch.empty(k, N, dtype=torch.float64, device="cuda")
    opts = _tps().default_opts()
    for key, v in kw.items():
        setattr(opts, key, v)
    lam, st = ctx.solve(k, parity, tol, block, ev, opts=opts)
    return lam, host(ev), st


def _sign_fix(X):
    X = X.copy()
    for i in range(X.shape[0]):
        j = np.argmax(np.abs(X[i]))
        if X[i, j] < 0:
            X[i] = -X[i]
    return X


def _check_vectors(P, lam, X, parity_sign=None, tol_res=1e-11):
    assert np.allclose(np.linalg.norm(X, axis=1), 1.0, atol=1e-12)
    for i in range(X.shape[0]):
        j = np.argmax(np.abs(X[i]))
        assert X[i, j] > 0
    res = residual_norms(P, X, lam)
    assert res.max() <= tol_res * P.norm_estimate(), res.max() / P.norm_estimate()
    if parity_sign is not None:
        assert np.max(np.abs(reflect_x(P, X) - parity_sign * X)) <= 1e-12
    return res


def test_solve_workload_1d_n64():
    require_gpu()
    tps = _tps()
    w = WORKLOADS["1d_n64"]
    P = problem_1d(w.M, w.m, w.hbar, w.n, w.L, w.v0, w.sigma)
    ctx = make_ctx_1d(w.M, w.m, w.n, w.L, w.v0, w.sigma)
    lam, X, st = _solve(ctx, w.k, tps.X_EVEN, w.block)
    ref, Xr = lowest_dense(P, w.k, O_EVEN)
    assert np.max(np.abs(lam - ref) / np.abs(ref)) <= 1e-10
    _check_vectors(P, lam, X, parity_sign=1.0)
    gaps = np.diff(all_eigenvalues_dense(P, O_EVEN)[: w.k + 1])
    Xr = _sign_fix(Xr)
    for i in range(w.k):
        if gaps[i] > 1e-6 and (i == 0 or gaps[i - 1] > 1e-6):
            assert np.linalg.norm(X[i] - Xr[i]) <= 1e-8
    assert st.n_converged == w.k and st.outer_iters > 0 and st.h_applies > 0


@pytest.mark.parametrize("parity", [0, 1, 2])
def test_solve_brute_force_small(parity):
    require_gpu()
    n, L = (16, 16), (6.0, 6.0)
    P = problem_1d(20.0, 1.0, 1.0, n, L, 1.0, 1.0)
    ctx = make_ctx_1d(20.0, 1.0, n, L, 1.0, 1.0)
    lam, X, st = _solve(ctx, 5, parity, 3)
    full = all_eigenvalues_dense(P, [O_ANY, O_EVEN, O_ODD][parity])
    assert np.max(np.abs(lam - full[:5]) / np.abs(full[:5])) <= 1e-10
    _check_vectors(P, lam, X, parity_sign=[None, 1.0, -1.0][parity])


def test_solve_constant_potential_closed_form():
    # V = -1: levels -1 + |a_x|(k pi/L_x)^2 + |a_y|(l pi/L_y)^2, degenerate pairs in l
    require_gpu()
    tps = _tps()
    n, L = (32, 24), (5.0, 4.0)
    ax, ay, _ = coefficients_from_masses(20.0, 1.0, 1.0)
    V = np.full(n, -1.0)
    kx = np.arange(0, n[0] // 2 + 1) * np.pi / L[0]
    ky = np.concatenate([[0], np.repeat(np.arange(1, n[1] // 2), 2), [n[1] // 2]]) * np.pi / L[1]
    lev = np.sort((-1.0 - ax * kx[:, None] ** 2 - ay * ky[None, :] ** 2).ravel())
    k = 7   # closes the cluster: lev[6] < lev[7]
    assert lev[k] - lev[k - 1] > 1e-6
    P = Problem((ax, ay), n, L, V)
    ctx = make_ctx_1d(20.0, 1.0, n, L, 0, 1, V=V)
    lam, X, st = _solve(ctx, k, tps.X_EVEN, 4)
    assert np.max(np.abs(lam - lev[:k]) / np.abs(lev[:k])) <= 1e-10
    _check_vectors(P, lam, X, parity_sign=1.0)


def test_solve_harmonic_closed_form():
    require_gpu()
    tps = _tps()
    M, m = 20.0, 1.0
    ax, ay, _ = coefficients_from_masses(M, m, 1.0)
    mu_x, mu_y = -1 / (2 * ax), -1 / (2 * ay)
    wx, wy = 1 / mu_x, 1 / mu_y
    n, L = (64, 64), (10.0, 10.0)
    x = -10.0 + np.arange(64) * 20.0 / 64
    V = 0.5 * mu_x * wx ** 2 * x[:, None] ** 2 + 0.5 * mu_y * wy ** 2 * x[None, :] ** 2
    ctx = make_ctx_1d(M, m, n, L, 0, 1, V=V)
    lam, X, st = _solve(ctx, 6, tps.X_EVEN, 3)
    levels = np.array(sorted((p + 0.5) * wx + (q + 0.5) * wy for p in range(0, 40, 2) for q in range(10))[:6])
    assert np.max(np.abs(lam - levels) / levels) <= 1e-10


@pytest.mark.parametrize("use_prec,block,prec_dtype,h_dtype", [(0, 4, 1, 1), (1, 1, 1, 1), (0, 1, 1, 1),
                                                         (1, 4, 0, 0), (1, 4, 1, 0)])
def test_solve_variants_agree(use_prec, block, prec_dtype, h_dtype):
    # FP64-only and mixed-precision solvers, no-prec-JDQR and the single-vector JDQR
    # no-prec-JDQR and the paper's single-vector JDQR reach the same eigenpairs
    require_gpu()
    n, L = (48, 48), (15.0, 15.0)
    P = problem_1d(20.0, 1.0, 1.0, n, L, 1.0, 1.0)
    ctx = make_ctx_1d(20.0, 1.0, n, L, 1.0, 1.0)
    lam, X, st = _solve(ctx, 3, 1, block, use_prec=use_prec, max_outer=3000,
                        inner_steps=20 if not use_prec else 10, prec_dtype=prec_dtype,
                        h_dtype=h_dtype)
    ref, _ = lowest_dense(P, 3, O_EVEN)
    assert np.max(np.abs(lam - ref) / np.abs(ref)) <= 1e-10
    _check_vectors(P, lam, X, parity_sign=1.0)


def test_warm_start_converges_at_once():
    require_gpu()
    tps = _tps()
    w = WORKLOADS["1d_n64"]
    ctx = make_ctx_1d(w.M, w.m, w.n, w.L, w.v0, w.sigma)
    lam, X, st = _solve(ctx, 4, tps.X_EVEN, 4)
    ev = torch.empty(4, ctx.info()[0], dtype=torch.float64, device="cuda")
    o = tps.default_opts()
    o.guard = 0          # the start block already holds the answer
    lam2, st2 = ctx.solve(4, tps.X_EVEN, 1e-12, 4, ev, x0=dev(X), opts=o)
    assert st2.outer_iters <= 2
    assert np.max(np.abs(lam2 - lam) / np.abs(lam)) <= 1e-12


def test_not_converged_and_bad_args():
    require_gpu()
    tps = _tps()
    ctx = make_ctx_1d(20.0, 1.0, (32, 32), (10.0, 10.0), 1.0, 1.0)
    ev = torch.empty(3, ctx.info()[0], dtype=torch.float64, device="cuda")
    o = tps.default_opts()
    o.max_outer = 1
    with pytest.raises(tps.TpsError) as e:
        ctx.solve(3, 1, 1e-12, 3, ev, opts=o)
    assert e.value.status == tps.ERR_NOT_CONVERGED
    with pytest.raises(tps.TpsError) as e:
        ctx.solve(3, 7, 1e-12, 3, ev)
    assert e.value.status == tps.ERR_INVALID_ARG
    c2 = make_ctx_2d(20.0, 1.0, (8, 8, 8, 8), (4.0,) * 4, 1.0, 1.0)
    ev2 = torch.empty(1, c2.info()[0], dtype=torch.float64, device="cuda")
    with pytest.raises(tps.TpsError):
        c2.solve(1, tps.X_EVEN, 1e-12, 1, ev2)


def test_solve_workload_1d_n512_full_size():
    require_gpu()
    tps = _tps()
    w = WORKLOADS["1d_n512"]
    with open(os.path.join(GOLD, "evals_1d_n512.json")) as f:
        gold = json.load(f)
    _, _, mu_hl = coefficients_from_masses(w.M, w.m, w.hbar)
    v0 = tps.two_body_v0(1, mu_hl, w.hbar, w.E0, tps.GAUSS, w.sigma, w.n[1], w.L[1])
    assert v0 == pytest.approx(gold["v0"], rel=1e-11)
    ctx = make_ctx_1d(w.M, w.m, w.n, w.L, v0, w.sigma)
    lam, X, st = _solve(ctx, w.k, tps.X_EVEN, w.block)
    ref = np.array(gold["evals"])
    assert np.max(np.abs(lam - ref) / np.abs(ref)) <= 1e-10
    P = problem_1d(w.M, w.m, w.hbar, w.n, w.L, gold["v0"], w.sigma)
    res = _check_vectors(P, lam, X, parity_sign=1.0)
    # Kato-Temple with the oracle's spectrum: each pair certified far below 1e-10 relative
    weyl, kt = certify(lam, res, ref)
    assert np.all(kt <= 1e-12 * np.abs(lam))


@pytest.mark.parametrize("parity,key,k,seed", [(1, "bosons", 3, 12345), (2, "fermions", 2, 12345),
                                               (1, "bosons", 3, 1), (1, "bosons", 3, 2),
                                               (1, "bosons", 3, 3)])
def test_table1_physics_on_gpu(parity, key, k, seed):
    # Table 1 (Sec. 5.1), E0 = 0.1, M/m = 20, heavy-light units, converged grid
    require_gpu()
    tps = _tps()
    with open(os.path.join(GOLD, "table1.json")) as f:
        row = json.load(f)["rows"][0]
    v0 = tps.two_body_v0(1, 1.0, 1.0, row["E0"], tps.GAUSS, 1.0, 512, 100.0)
    assert abs(v0 - row["v0"]) <= 0.5e-8 + 1e-10
    ctx = make_ctx_1d(None, None, (288, 288), (60.0, 60.0), v0, 1.0, alpha=20.0)
    lam, X, st = _solve(ctx, k, parity, k, seed=seed)   # random starts must not skip a state
    assert np.max(np.abs(lam / row["E0"] - np.array(row[key][:k]))) <= 1.0e-8


def test_solve_2d_small_against_oracle():
    require_gpu()
    tps = _tps()
    with open(os.path.join(GOLD, "evals_2d_n16.json")) as f:
        gold = json.load(f)
    ctx = make_ctx_2d(gold["M"], gold["m"], gold["n"], gold["L"], gold["v0"], gold["sigma"])
    lam, X, st = _solve(ctx, 4, tps.ANY, 4)
    ref = np.array(gold["evals"])
    assert np.max(np.abs(lam - ref) / np.abs(ref)) <= 1e-10
    P = problem_2d(gold["M"], gold["m"], 1.0, gold["n"], gold["L"], gold["v0"], gold["sigma"])
    _check_vectors(P, lam, X)


@pytest.mark.parametrize("h64_dtype", [0, 2])
def test_solve_2d_n24_against_oracle(h64_dtype):
    """The 2D solve at 24^4 (331,776 unknowns, between the brute-force-checked 16^4 and the
    48^4 workload): the 4 lowest eigenvalues against the oracle's LOBPCG values, with the
    FP64 H-applies on the FMA pipe and on the tensor cores."""
    require_gpu()
    tps = _tps()
    with open(os.path.join(GOLD, "evals_2d_n24.json")) as f:
        gold = json.load(f)
    ctx = make_ctx_2d(gold["M"], gold["m"], gold["n"], gold["L"], gold["v0"], gold["sigma"])
    lam, X, st = _solve(ctx, 4, tps.ANY, 8, h64_dtype=h64_dtype)
    ref = np.array(gold["evals"])
    assert np.max(np.abs(lam - ref) / np.abs(ref)) <= 1e-10


def test_solve_workload_2d_n48_certified():
    # full 2D workload: certified by the oracle's residual (Weyl bound) at 1e-10 relative
    require_gpu()
    tps = _tps()
    w = WORKLOADS["2d_n48"]
    ctx = make_ctx_2d(w.M, w.m, w.n, w.L, w.v0, w.sigma)
    lam, X, st = _solve(ctx, w.k, tps.ANY, w.block)
    P = problem_2d(w.M, w.m, w.hbar, w.n, w.L, w.v0, w.sigma)
    res = _check_vectors(P, lam, X)
    assert np.all(res <= 1e-10 * np.abs(lam))


@pytest.mark.parametrize("h_dtype,h64_dtype", [(0, 0), (0, 2), (1, 0), (1, 2)])
def test_full_size_fp64_and_mixed_agree(h_dtype, h64_dtype):
    # the FP64-only solver and the mixed-precision one on the 1d_n512 workload, with the
    # FP64 H-applies on the FMA pipe or the tensor cores
    require_gpu()
    tps = _tps()
    w = WORKLOADS["1d_n512"]
    with open(os.path.join(GOLD, "evals_1d_n512.json")) as f:
        gold = json.load(f)
    ctx = make_ctx_1d(w.M, w.m, w.n, w.L, gold["v0"], w.sigma)
    lam, X, st = _solve(ctx, w.k, tps.X_EVEN, w.block, h_dtype=h_dtype, h64_dtype=h64_dtype,
                        timing=1)
    assert st.gram_launches > 0 and st.gram_ms > 0 and st.upd_launches > 0
    ref = np.array(gold["evals"])
    assert np.max(np.abs(lam - ref) / np.abs(ref)) <= 1e-10
    if h_dtype == 1:
        assert st.h32_launches > 0 and st.h32_flops > 0
    else:
        assert st.h32_launches == 0


def test_new_potential_on_a_used_context_matches_a_fresh_context():
    # changing the potential keeps the context's sector operators (mode matrices,
    # eigenbases, tensor-core slices) and refreshes only their V
    require_gpu()
    tps = _tps()
    w = WORKLOADS["1d_n64"]
    ctx = make_ctx_1d(w.M, w.m, w.n, w.L, w.v0, w.sigma)
    lam_a, _, _ = _solve(ctx, w.k, tps.X_EVEN, w.block)
    ctx.set_pair_potential(tps.GAUSS, 1.7 * w.v0, 0.8)
    lam_b, Xb, _ = _solve(ctx, w.k, tps.X_EVEN, w.block)
    fresh = make_ctx_1d(w.M, w.m, w.n, w.L, 1.7 * w.v0, 0.8)
    lam_f, _, _ = _solve(fresh, w.k, tps.X_EVEN, w.block)
    assert np.max(np.abs(lam_b - lam_f) / np.abs(lam_f)) <= 1e-11
    assert np.max(np.abs(lam_b - lam_a) / np.abs(lam_a)) > 1e-3
    P = problem_1d(w.M, w.m, w.hbar, w.n, w.L, 1.7 * w.v0, 0.8)
    ref, _ = lowest_dense(P, w.k, O_EVEN)
    assert np.max(np.abs(lam_b - ref) / np.abs(ref)) <= 1e-10
    # an explicit potential array (host path) on the same context
    ctx.set_potential(P.V.ravel())
    lam_c, _, _ = _solve(ctx, w.k, tps.X_EVEN, w.block)
    assert np.max(np.abs(lam_c - ref) / np.abs(ref)) <= 1e-10
    ctx.close()
    fresh.close()


@pytest.mark.parametrize("rr_method,refine_max", [(0, 0), (1, 0), (0, 1)])
def test_rayleigh_ritz_methods_agree_full_size(rr_method, refine_max):
    # the Rayleigh-Ritz eigensolver by FP32 Jacobi + FP64 refinement (default), by FP64
    # cyclic Jacobi, and with the refinement cut to one iteration so that most solves fall
    # back to the FP64 Jacobi inside the same launch: the same eigenpairs on the 1d_n512
    # workload, every pair certified by the oracle's residual
    require_gpu()
    tps = _tps()
    w = WORKLOADS["1d_n512"]
    with open(os.path.join(GOLD, "evals_1d_n512.json")) as f:
        gold = json.load(f)
    ctx = make_ctx_1d(w.M, w.m, w.n, w.L, gold["v0"], w.sigma)
    lam, X, st = _solve(ctx, w.k, tps.X_EVEN, w.block, rr_method=rr_method,
                        rr_refine_max=refine_max)
    ref = np.array(gold["evals"])
    assert np.max(np.abs(lam - ref) / np.abs(ref)) <= 1e-10
    P = problem_1d(w.M, w.m, w.hbar, w.n, w.L, gold["v0"], w.sigma)
    res = _check_vectors(P, lam, X, parity_sign=1.0)
    weyl, kt = certify(lam, res, ref)
    assert np.all(kt <= 1e-12 * np.abs(lam))
    if rr_method == tps.RR_JACOBI64:
        assert st.rr_mixed_calls == 0 and st.jacobi_calls == st.outer_iters
    else:
        assert st.rr_mixed_calls == st.outer_iters and st.rr_fp32_solves >= st.rr_mixed_calls
        if refine_max == 1:
            assert st.rr_fallbacks > 0 and st.jacobi_calls == st.rr_fallbacks
        else:
            assert st.rr_fallbacks == 0 and st.jacobi_calls == 0
            assert st.rr_refine_iters >= st.rr_mixed_calls
    ctx.close()


def test_tf32_preconditioner_solve_full_size():
    # the solver with the TF32 tensor-core preconditioner: the same certified eigenpairs on
    # the 1d_n512 workload, with about as many H applications as the FP32 preconditioner
    require_gpu()
    tps = _tps()
    w = WORKLOADS["1d_n512"]
    with open(os.path.join(GOLD, "evals_1d_n512.json")) as f:
        gold = json.load(f)
    ctx = make_ctx_1d(w.M, w.m, w.n, w.L, gold["v0"], w.sigma)
    lam32, _, st32 = _solve(ctx, w.k, tps.X_EVEN, w.block, prec_dtype=tps.F32)
    lam, X, st = _solve(ctx, w.k, tps.X_EVEN, w.block, prec_dtype=tps.TF32_TC)
    ctx.device_status()
    ref = np.array(gold["evals"])
    assert np.max(np.abs(lam - ref) / np.abs(ref)) <= 1e-10
    P = problem_1d(w.M, w.m, w.hbar, w.n, w.L, gold["v0"], w.sigma)
    res = _check_vectors(P, lam, X, parity_sign=1.0)
    weyl, kt = certify(lam, res, ref)
    assert np.all(kt <= 1e-12 * np.abs(lam))
    assert st.h_applies <= 1.25 * st32.h_applies, (st.h_applies, st32.h_applies)
    ctx.close()


def test_correction_products_fp32_and_fp64_agree_full_size():
    # the correction solve's Gram/update products in FP32 arithmetic (default) or FP64: the
    # same certified eigenpairs on the 1d_n512 workload and about as many H applications
    require_gpu()
    tps = _tps()
    w = WORKLOADS["1d_n512"]
    with open(os.path.join(GOLD, "evals_1d_n512.json")) as f:
        gold = json.load(f)
    ctx = make_ctx_1d(w.M, w.m, w.n, w.L, gold["v0"], w.sigma)
    P = problem_1d(w.M, w.m, w.hbar, w.n, w.L, gold["v0"], w.sigma)
    ref = np.array(gold["evals"])
    applies = {}
    for cd in (tps.F32, tps.F64):
        lam, X, st = _solve(ctx, w.k, tps.X_EVEN, w.block, correction_dtype=cd)
        assert np.max(np.abs(lam - ref) / np.abs(ref)) <= 1e-10
        res = _check_vectors(P, lam, X, parity_sign=1.0)
        weyl, kt = certify(lam, res, ref)
        assert np.all(kt <= 1e-12 * np.abs(lam))
        applies[cd] = st.h_applies
    assert applies[tps.F32] <= 1.25 * applies[tps.F64], applies
    ctx.close()


@pytest.mark.parametrize("parity", [0, 1, 2])
def test_split_updates_brute_force_small(parity):
    # the outer iteration's block updates as digit-split tensor-core products
    # (update_dtype = F64_TC): eigenvalues of a 16 x 16 problem against dense brute force
    require_gpu()
    tps = _tps()
    n, L = (16, 16), (6.0, 6.0)
    P = problem_1d(20.0, 1.0, 1.0, n, L, 1.0, 1.0)
    ctx = make_ctx_1d(20.0, 1.0, n, L, 1.0, 1.0)
    lam, X, st = _solve(ctx, 5, parity, 3, update_dtype=tps.F64_TC)
    full = all_eigenvalues_dense(P, [O_ANY, O_EVEN, O_ODD][parity])
    assert np.max(np.abs(lam - full[:5]) / np.abs(full[:5])) <= 1e-10
    _check_vectors(P, lam, X, parity_sign=[None, 1.0, -1.0][parity])
    ctx.close()


def test_split_updates_full_size():
    # update_dtype = F64_TC on the 1d_n512 workload: the same certified eigenpairs
    require_gpu()
    tps = _tps()
    w = WORKLOADS["1d_n512"]
    with open(os.path.join(GOLD, "evals_1d_n512.json")) as f:
        gold = json.load(f)
    ctx = make_ctx_1d(w.M, w.m, w.n, w.L, gold["v0"], w.sigma)
    P = problem_1d(w.M, w.m, w.hbar, w.n, w.L, gold["v0"], w.sigma)
    ref = np.array(gold["evals"])
    lam, X, st = _solve(ctx, w.k, tps.X_EVEN, w.block, update_dtype=tps.F64_TC)
    assert np.max(np.abs(lam - ref) / np.abs(ref)) <= 1e-10
    res = _check_vectors(P, lam, X, parity_sign=1.0)
    weyl, kt = certify(lam, res, ref)
    assert np.all(kt <= 1e-12 * np.abs(lam))
    ctx.close()
