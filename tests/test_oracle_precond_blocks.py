"""Pins for oracle.precond and oracle.blocks."""
import numpy as np
import pytest

from oracle.hamiltonian import problem_1d, problem_2d, Problem
from oracle.precond import apply_dense, apply_sylvester, kinetic_residual
from oracle import blocks


def test_sylvester_equals_dense_solve():
    P = problem_1d(20.0, 1.0, 1.0, (12, 10), (4.0, 5.0), 1.0, 1.0)
    r = np.random.default_rng(0).uniform(-1, 1, size=(2, P.N))
    for theta in (-0.3, -2.0):
        a = apply_dense(P, r, theta)
        b = apply_sylvester(P, r, theta)
        assert np.max(np.abs(a - b)) <= 1e-12 * np.abs(a).max()


def test_exact_inverse_for_constant_potential():
    # V = c: H - theta' = T - (theta' - c), so the preconditioner at theta = theta' - c inverts it
    n = (16, 12)
    P0 = problem_1d(20.0, 1.0, 1.0, n, (4.0, 5.0), 1.0, 1.0)
    c, th = -1.0, -1.4
    P = Problem(P0.a, n, P0.L, np.full(n, c))
    psi = np.random.default_rng(1).uniform(-1, 1, size=(1, P.N))
    w = apply_sylvester(P, P.apply_kron(psi, th), th - c)
    assert np.max(np.abs(w - psi)) <= 1e-12
    assert kinetic_residual(P, w, P.apply_kron(psi, th), th - c) <= 1e-12


def test_dense_2d_against_residual():
    P = problem_2d(20.0, 1.0, 1.0, (4, 4, 4, 4), (2.0, 2.0, 3.0, 3.0), 1.0, 1.0)
    r = np.random.default_rng(2).uniform(-1, 1, size=(1, P.N))
    w = apply_dense(P, r, -0.5)
    assert kinetic_residual(P, w, r, -0.5) <= 1e-12


def _sym(n, seed):
    A = np.random.default_rng(seed).standard_normal((n, n))
    return 0.5 * (A + A.T)


def test_rayleigh_ritz_full_space_is_exact():
    A = _sym(20, 0)
    V = np.linalg.qr(np.random.default_rng(1).standard_normal((20, 20)))[0]
    th, Y, X, R = blocks.rayleigh_ritz(V, A @ V)
    assert np.allclose(th, np.linalg.eigvalsh(A), atol=1e-12)
    assert np.max(np.abs(R)) <= 1e-12


def test_expansion_step_and_projection():
    rng = np.random.default_rng(3)
    Q = np.linalg.qr(rng.standard_normal((30, 5)))[0]
    T = rng.standard_normal((30, 3))
    Z = blocks.orthonormal_complement_step(Q, T)
    assert np.allclose(Z.T @ Z, np.eye(3), atol=1e-13)
    assert np.max(np.abs(Q.T @ Z)) <= 1e-13
    # span(Q, Z) contains T
    W = np.concatenate([Q, Z], axis=1)
    assert np.max(np.abs(T - W @ (W.T @ T))) <= 1e-12
    x = rng.standard_normal(30)
    assert np.max(np.abs(Q.T @ blocks.project_out(Q, x))) <= 1e-13


def test_correction_and_projected_preconditioner():
    rng = np.random.default_rng(4)
    A = _sym(24, 5)
    w, U = np.linalg.eigh(A)
    q = U[:, 0] + 1e-3 * rng.standard_normal(24)
    q /= np.linalg.norm(q)
    theta = q @ A @ q
    r = A @ q - theta * q
    Qt = q[:, None]
    dq = blocks.correction_exact(A, Qt, theta, r)
    Pm = np.eye(24) - Qt @ Qt.T
    assert abs(q @ dq) <= 1e-13
    assert np.max(np.abs(Pm @ (A - theta * np.eye(24)) @ Pm @ dq + r)) <= 1e-11
    # with K = A - theta exactly, the projected preconditioner inverts the projected operator
    Kinv = lambda y: np.linalg.solve(A - theta * np.eye(24) + 0.0, y)
    t = Pm @ rng.standard_normal(24)
    y = Pm @ (A - theta * np.eye(24)) @ Pm @ t
    z = blocks.projected_preconditioner(Kinv, Qt, y)
    assert np.max(np.abs(z - t)) <= 1e-8 * np.linalg.norm(t)
    assert abs(q @ z) <= 1e-10


def test_gmres_full_dimension_is_exact():
    rng = np.random.default_rng(6)
    A = _sym(12, 7) + 12 * np.eye(12)
    b = rng.standard_normal(12)
    x, res = blocks.gmres(lambda v: A @ v, b, 12)
    assert np.allclose(x, np.linalg.solve(A, b), atol=1e-10)
    assert all(res[i + 1] <= res[i] + 1e-14 for i in range(len(res) - 1))
