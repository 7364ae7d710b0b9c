"""Pins for oracle.mlp (the warm-start network's CPU oracle): every function against
something other than itself -- finite differences, scalar loops, closed forms."""
import math

import numpy as np
import pytest
from scipy.stats import norm

from oracle import mlp

RNG = np.random.Generator(np.random.PCG64(5))


def _tiny(hidden=5, px=3, py=4, rank=2):
    dims = mlp.layer_dims(px, py, rank, hidden)
    params = RNG.normal(size=mlp.n_params(dims)) * 0.7
    return dims, params


def test_gelu_is_z_times_normal_cdf_and_grad_matches_difference():
    z = np.linspace(-6, 6, 121)
    assert np.allclose(mlp.gelu(z), z * norm.cdf(z), rtol=0, atol=1e-14)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(z), fd, rtol=0, atol=1e-8)


def test_forward_matches_scalar_loops():
    dims, params = _tiny()
    X = RNG.normal(size=(3, 4))
    out, _ = mlp.forward(params, dims, X)
    # the layer layout written out with scalar loops: W_l[i][j] at offset + i*out + j
    off = 0
    a = [list(r) for r in X]
    for l in range(4):
        n_in, n_out = dims[l], dims[l + 1]
        W = params[off: off + n_in * n_out]
        b = params[off + n_in * n_out: off + n_in * n_out + n_out]
        off += n_in * n_out + n_out
        new = []
        for r in a:
            row = []
            for j in range(n_out):
                z = b[j] + sum(r[i] * W[i * n_out + j] for i in range(n_in))
                row.append(z * 0.5 * (1 + math.erf(z / math.sqrt(2))) if l < 3 else z)
            new.append(row)
        a = new
    assert np.allclose(out, np.array(a), rtol=1e-13, atol=1e-13)


def test_backward_matches_central_differences():
    dims, params = _tiny()
    px, py, rank = 3, 4, 2
    X = RNG.normal(size=(4, 4))
    T = RNG.normal(size=(4, px, py))
    _, g = mlp.loss_and_grad(params, dims, X, T, rank, px, py)
    h = 1e-6
    idx = RNG.choice(params.size, size=40, replace=False)
    for i in idx:
        p1, p2 = params.copy(), params.copy()
        p1[i] += h
        p2[i] -= h
        f1, _ = mlp.loss_and_grad(p1, dims, X, T, rank, px, py)
        f2, _ = mlp.loss_and_grad(p2, dims, X, T, rank, px, py)
        fd = (f1 - f2) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, g[i])


def test_cosine_loss_special_cases():
    px, py, rank = 3, 2, 1
    C = RNG.normal(size=(1, rank, px))
    D = RNG.normal(size=(1, rank, py))
    o = np.concatenate([C.reshape(1, -1), D.reshape(1, -1)], axis=1)
    P = np.einsum("sra,srb->sab", C, D)
    assert mlp.cosine_loss(o, P, rank, px, py)[0] == pytest.approx(0.0, abs=1e-14)
    assert mlp.cosine_loss(o, -3.0 * P, rank, px, py)[0] == pytest.approx(0.0, abs=1e-14)
    # a target orthogonal to P
    Tp = RNG.normal(size=P.shape)
    Tp -= np.sum(Tp * P) / np.sum(P * P) * P
    assert mlp.cosine_loss(o, Tp, rank, px, py)[0] == pytest.approx(1.0, abs=1e-12)


def test_adam_first_step_is_lr_times_sign():
    g = np.array([3.0, -0.5, 1e-3])
    w, m, v = mlp.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=1e-12)
    assert np.allclose(w, -0.01 * np.sign(g), rtol=1e-9)


@pytest.mark.parametrize("n,na,kind", [(32, 16, 0), (32, 31, 1), (48, 10, 1)])
def test_mode_matrices_orthonormal(n, na, kind):
    M = mlp.mode_matrix(kind, n, na)
    assert np.allclose(M.T @ M, np.eye(na), atol=1e-13)
    if kind == 0:   # even under x -> -x on the grid: j -> (n - j) mod n
        refl = (-np.arange(n)) % n
        assert np.allclose(M[refl], M, atol=1e-13)


def test_project_and_assemble_round_trip():
    nx, ny, px, py, rank = 24, 20, 5, 6, 2
    C = RNG.normal(size=(2, rank, px))
    D = RNG.normal(size=(2, rank, py))
    o = np.concatenate([C.reshape(2, -1), D.reshape(2, -1)], axis=1)
    psi = mlp.assemble(o, rank, px, py, nx, ny)
    T = mlp.project(psi, nx, ny, px, py)
    assert np.allclose(T, np.einsum("sra,srb->sab", C, D), atol=1e-12)
    # a single product of modes projects onto one coefficient
    Phi, Chi = mlp.mode_matrix(0, nx, px), mlp.mode_matrix(1, ny, py)
    one = np.outer(Phi[:, 3], Chi[:, 4]).ravel()[None]
    T1 = mlp.project(one, nx, ny, px, py)[0]
    E = np.zeros((px, py))
    E[3, 4] = 1.0
    assert np.allclose(T1, E, atol=1e-13)


def test_features_are_the_stated_map():
    X = mlp.features(40.0, math.e ** 5, 2.0, 8)
    assert np.allclose(X, [[1.0, 1.0, 1.0, 1.0]], atol=1e-15)


def test_mode_matrix_2d_is_the_product_basis():
    # pinned to the modes written out from their formulas (not through mode_matrix):
    # F_0 = 1, F_1 = cos(t), F_2 = sin(t), F_3 = cos(2t), ... with t = pi x / L, x_j = -L + 2Lj/n
    n1, n2, q = 12, 10, 4
    def raw(a, n):
        t = 2.0 * np.pi * np.arange(n) / n - np.pi
        f = (a + 1) // 2
        return np.ones(n) if a == 0 else (np.cos(f * t) if a % 2 else np.sin(f * t))
    M = mlp.mode_matrix_2d(n1, n2, q)
    assert M.shape == (n1 * n2, q * q)
    assert np.allclose(M.T @ M, np.eye(q * q), atol=1e-13)
    for a1, a2 in ((0, 0), (1, 2), (3, 0), (2, 3)):
        g = np.outer(raw(a1, n1), raw(a2, n2)).ravel()
        assert np.allclose(M[:, a1 * q + a2], g / np.linalg.norm(g), atol=1e-14)


def test_project_and_assemble_2d():
    n, px, py, rank = (8, 6, 10, 6), 9, 16, 3
    C = RNG.normal(size=(2, rank, px))
    D = RNG.normal(size=(2, rank, py))
    o = np.concatenate([C.reshape(2, -1), D.reshape(2, -1)], axis=1)
    psi = mlp.assemble_2d(o, rank, px, py, n)
    assert psi.shape == (2, int(np.prod(n)))
    assert np.allclose(mlp.project_2d(psi, n, px, py), np.einsum("sra,srb->sab", C, D),
                       atol=1e-12)
    # a separable product cos(x1) sin(x2) * cos(2 y1) projects onto exactly one coefficient,
    # at (a1 q + a2, b1 q + b2) = (1*3 + 2, 3*4 + 0), with the product of the grid norms
    t = [2.0 * np.pi * np.arange(k) / k - np.pi for k in n]
    f = np.einsum("i,j,k,l->ijkl", np.cos(t[0]), np.sin(t[1]), np.cos(2 * t[2]),
                  np.ones(n[3]))
    T = mlp.project_2d(f.ravel()[None], n, px, py)[0]
    E = np.zeros((px, py))
    E[5, 12] = np.sqrt(n[0] / 2 * n[1] / 2 * n[2] / 2 * n[3])
    assert np.allclose(T, E, atol=1e-12)
    with pytest.raises(ValueError):
        mlp.project_2d(psi, n, 8, py)
