"""Learned warm start: the network, loss, optimiser and grid maps in plain NumPy FP64
(oracle; test infrastructure).

Definitions (the model of the warm-start extension; the paper's starting point is the
homotopy restart of Sec. 5.2 and the low-rank outlook of Sec. 6):

* features f(M/m, v0, sigma, state) = (ln(M/m)/ln 40, ln(v0)/5, ln(sigma)/ln 2, state/8);
* layers l = 0..3 with widths 4, H, H, H, R(px+py); z_l = a_l W_l + b_l, a_{l+1} = GELU(z_l)
  for l < 3 and the output o = z_3; GELU(z) = z Phi(z) with Phi the standard normal CDF;
* parameters in one array: per layer W_l (row-major [in][out]) then b_l;
* the output row o = (C, D), C = o[:R px] as R x px, D = o[R px:] as R x py, P = C^T D;
* loss per sample 1 - <P,T>^2 / (|P|^2 |T|^2), mean over the batch;
* Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
  w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps);
* grid maps: Phi[x][a] = cos(a pi x / L) sampled at x_j = -L + 2Lj/n and scaled to unit
  norm over the grid, Chi[y][b] the real Fourier modes 1, cos, sin, cos 2, sin 2, ... likewise;
  targets T = Phi^T psi Chi, predictions psi = Phi P Chi^T;
* 2D grid maps (psi laid out [x1][x2][y1][y2]): the same matrix form with psi a
  (n_x1 n_x2) x (n_y1 n_y2) matrix, Phi[(x1,x2)][(a1,a2)] = F_a1(x1) F_a2(x2) over the first
  q_x real Fourier modes F of each Cartesian component (px = q_x^2, a = a1 q_x + a2) and
  Chi likewise over y (py = q_y^2): products of unit-norm columns, so unit norm again.

Backpropagation is written out by hand (chain rule through each layer); tests pin it
to central finite differences of the forward pass.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

N_LAYERS = 4


def layer_dims(px: int, py: int, rank: int, hidden: int):
    return [4, hidden, hidden, hidden, rank * (px + py)]


def unpack(params: np.ndarray, dims):
    """List of (W, b) views into the flat parameter array."""
    out, off = [], 0
    for l in range(N_LAYERS):
        n_in, n_out = dims[l], dims[l + 1]
        W = params[off: off + n_in * n_out].reshape(n_in, n_out)
        off += n_in * n_out
        b = params[off: off + n_out]
        off += n_out
        out.append((W, b))
    assert off == params.size
    return out


def n_params(dims) -> int:
    return sum(dims[l] * dims[l + 1] + dims[l + 1] for l in range(N_LAYERS))


def features(mass_ratio, v0, sigma, state) -> np.ndarray:
    mr, vv, sg, st = (np.atleast_1d(np.asarray(a, dtype=np.float64))
                      for a in (mass_ratio, v0, sigma, state))
    return np.stack([np.log(mr) / np.log(40.0), np.log(vv) / 5.0, np.log(sg) / np.log(2.0),
                     st / 8.0], axis=1)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def forward(params, dims, X):
    """Returns (output, cache) for a batch X [B, 4]."""
    layers = unpack(np.asarray(params, dtype=np.float64), dims)
    a = np.asarray(X, dtype=np.float64)
    acts, zs = [a], []
    for l, (W, b) in enumerate(layers):
        z = a @ W + b
        zs.append(z)
        a = gelu(z) if l < N_LAYERS - 1 else z
        acts.append(a)
    return a, (acts, zs, layers)


def split_output(o, rank, px, py):
    C = o[..., : rank * px].reshape(o.shape[:-1] + (rank, px))
    D = o[..., rank * px:].reshape(o.shape[:-1] + (rank, py))
    return C, D


def cosine_loss(o, T, rank, px, py):
    """Mean loss over the batch and dL/do (same shape as o)."""
    B = o.shape[0]
    C, D = split_output(o, rank, px, py)
    P = np.einsum("sra,srb->sab", C, D)
    T = np.asarray(T, dtype=np.float64).reshape(B, px, py)
    a = np.einsum("sab,sab->s", P, T)
    pp = np.einsum("sab,sab->s", P, P)
    tt = np.einsum("sab,sab->s", T, T)
    den = pp * tt
    loss = 1.0 - a * a / den
    dP = (-2.0 * a / den)[:, None, None] * T + (2.0 * a * a / (den * pp))[:, None, None] * P
    dP /= B
    dC = np.einsum("sab,srb->sra", dP, D)
    dD = np.einsum("sab,sra->srb", dP, C)
    do = np.concatenate([dC.reshape(B, -1), dD.reshape(B, -1)], axis=1)
    return loss.mean(), do


def loss_and_grad(params, dims, X, T, rank, px, py):
    """Mean loss and its gradient with respect to the flat parameter array."""
    o, (acts, zs, layers) = forward(params, dims, X)
    loss, dz = cosine_loss(o, T, rank, px, py)
    grads = []
    for l in range(N_LAYERS - 1, -1, -1):
        W, _ = layers[l]
        dW = acts[l].T @ dz
        db = dz.sum(axis=0)
        grads.append((dW, db))
        if l > 0:
            dz = (dz @ W.T) * gelu_grad(zs[l - 1])
    grads.reverse()
    flat = np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in grads])
    return loss, flat


def adam_step(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t >= 1); returns new (w, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    w = w - lr * (m / (1.0 - b1 ** t)) / (np.sqrt(v / (1.0 - b2 ** t)) + eps)
    return w, m, v


def mode_matrix(kind: int, n: int, na: int) -> np.ndarray:
    """n x na grid samples of the modes (kind 0: x-even cosines, 1: real Fourier), each
    column scaled to unit Euclidean norm over the grid."""
    t = 2.0 * np.pi * np.arange(n) / n - np.pi          # pi x / L on the grid
    cols = []
    for a in range(na):
        if kind == 0:
            c = np.cos(a * t)
        elif a == 0:
            c = np.ones(n)
        else:
            f = (a + 1) // 2
            c = np.cos(f * t) if a % 2 == 1 else np.sin(f * t)
        cols.append(c / np.linalg.norm(c))
    return np.stack(cols, axis=1)


def project(psi, nx, ny, px, py):
    """Targets T[v] = Phi^T psi_v Chi for psi [k, nx*ny]."""
    Phi, Chi = mode_matrix(0, nx, px), mode_matrix(1, ny, py)
    P = np.asarray(psi, dtype=np.float64).reshape(-1, nx, ny)
    return np.einsum("xa,vxy,yb->vab", Phi, P, Chi)


def assemble(o, rank, px, py, nx, ny):
    """Grid functions psi[v] = Phi (C^T D) Chi^T from network outputs o [k, R(px+py)]."""
    C, D = split_output(np.asarray(o, dtype=np.float64), rank, px, py)
    P = np.einsum("sra,srb->sab", C, D)
    Phi, Chi = mode_matrix(0, nx, px), mode_matrix(1, ny, py)
    return np.einsum("xa,sab,yb->sxy", Phi, P, Chi).reshape(len(o), nx * ny)


def mode_matrix_2d(n1: int, n2: int, q: int) -> np.ndarray:
    """(n1 n2) x q^2 samples of the product modes F_a1(x1) F_a2(x2) (real Fourier modes of
    each Cartesian component), row x1 n2 + x2, column a1 q + a2."""
    F1, F2 = mode_matrix(1, n1, q), mode_matrix(1, n2, q)
    out = np.empty((n1 * n2, q * q))
    for x1 in range(n1):
        for x2 in range(n2):
            for a1 in range(q):
                for a2 in range(q):
                    out[x1 * n2 + x2, a1 * q + a2] = F1[x1, a1] * F2[x2, a2]
    return out


def _side(p: int) -> int:
    q = int(round(np.sqrt(p)))
    if q * q != p:
        raise ValueError("2D grid maps need px and py to be perfect squares")
    return q


def project_2d(psi, n, px, py):
    """Targets T[v] = Phi^T psi_v Chi for 2D psi [k, n0 n1 n2 n3]."""
    Phi = mode_matrix_2d(n[0], n[1], _side(px))
    Chi = mode_matrix_2d(n[2], n[3], _side(py))
    P = np.asarray(psi, dtype=np.float64).reshape(-1, n[0] * n[1], n[2] * n[3])
    return np.einsum("xa,vxy,yb->vab", Phi, P, Chi)


def assemble_2d(o, rank, px, py, n):
    """2D grid functions psi[v] = Phi (C^T D) Chi^T from network outputs o [k, R(px+py)]."""
    C, D = split_output(np.asarray(o, dtype=np.float64), rank, px, py)
    P = np.einsum("sra,srb->sab", C, D)
    Phi = mode_matrix_2d(n[0], n[1], _side(px))
    Chi = mode_matrix_2d(n[2], n[3], _side(py))
    return np.einsum("xa,sab,yb->sxy", Phi, P, Chi).reshape(len(o), -1)
