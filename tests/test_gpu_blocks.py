"""GPU parity of the Jacobi-Davidson building blocks (Sec. 4.1) through the C ABI:
Gram matrices, block updates, the device Jacobi eigensolver, block orthonormalisation
and the preconditioned GMRES correction solve, against oracle.blocks definitions."""
import numpy as np
import pytest

from gpu_common import torch, require_gpu, make_ctx_1d, dev, host
from oracle import blocks
from oracle.hamiltonian import problem_1d, Problem
from oracle.precond import apply_dense
from paper_2111_02534_gb300.inputs import random_block

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    return make_ctx_1d(20.0, 1.0, (8, 8), (3.0, 3.0), 1.0, 1.0)


@pytest.mark.parametrize("nrows,p,q", [(131584, 24, 8), (1000003, 5, 1), (4097, 64, 64),
                                       (257, 1, 1), (0, 3, 2),
                                       # every register tile: 16x1, 8x1, 4x1, 2x1, 8x2, 4x2,
                                       # 2x2, operands swapped (p < q), ragged 4x4
                                       (50001, 13, 1), (30011, 7, 1), (20011, 3, 1),
                                       (9999, 2, 1), (70001, 7, 2), (4099, 3, 2), (777, 2, 2),
                                       (65537, 1, 5), (12345, 2, 11), (131584, 10, 8)])
def test_gram(ctx, nrows, p, q):
    A = random_block(p, nrows, 1)
    B = random_block(q, nrows, 2)
    G = torch.full((q, p), np.nan, dtype=torch.float64, device="cuda")   # column-major p x q
    ctx.gram(dev(A), p, dev(B), q, nrows, G)
    got = host(G).T
    ref = A @ B.T
    scale = max(1.0, np.sqrt(nrows))
    assert np.max(np.abs(got - ref)) <= 1e-14 * scale * max(1.0, np.abs(ref).max())


def _gram_bound(A, B):
    # the split Gram's error per entry: per 64-row block at most ~2^-53 (max|A_i| sum|B_j| +
    # sum|A_i| max|B_j|) (slack 4), plus the FP64 sum over the blocks and the reference's
    # rounding, at most (blocks + 2) 2^-53 sum |A_i| |B_j|
    p, n = A.shape
    q = B.shape[0]
    nb = (n + 63) // 64
    Ap = np.zeros((p, nb * 64))
    Bp = np.zeros((q, nb * 64))
    Ap[:, :n] = np.abs(A)
    Bp[:, :n] = np.abs(B)
    Ab, Bb = Ap.reshape(p, nb, 64), Bp.reshape(q, nb, 64)
    amax, asum = Ab.max(axis=2), Ab.sum(axis=2)    # p x nb
    bmax, bsum = Bb.max(axis=2), Bb.sum(axis=2)    # q x nb
    bound = 4 * 2.0 ** -53 * (amax @ bsum.T + asum @ bmax.T)
    return bound + (nb + 2) * 2.0 ** -53 * (np.abs(A) @ np.abs(B).T)


def _exact_gram(A, B):
    # the reference in the widest float numpy has (80-bit or 128-bit long double)
    return (A.astype(np.longdouble) @ B.astype(np.longdouble).T).astype(np.float64)


@pytest.mark.parametrize("nrows,p,q", [(131584, 24, 8), (131590, 36, 8), (100003, 64, 8),
                                       (70001, 8, 40), (1000, 17, 5), (200000, 48, 2),
                                       (777, 1, 1), (65, 16, 3), (64, 3, 64), (0, 5, 5)])
def test_gram_tc(ctx, nrows, p, q):
    # digit-split Gram: ragged last 64-row block, one to four 16-column m tiles, p < q
    # (operands swapped, result stored transposed), tiny and empty inputs; against the
    # exact product within the scheme's bound, against the FMA-pipe Gram, and the same bits
    # on a second call
    from paper_2111_02534_gb300 import tps
    A = random_block(p, max(nrows, 1), 21)[:, :nrows]
    B = random_block(q, max(nrows, 1), 22)[:, :nrows]
    G = torch.full((q, p), np.nan, dtype=torch.float64, device="cuda")
    dA, dB = dev(np.ascontiguousarray(A)), dev(np.ascontiguousarray(B))
    ctx.gram(dA, p, dB, q, nrows, G, dtype=tps.F64_TC)
    got = host(G).T
    if nrows == 0:
        assert np.all(got == 0.0)
        return
    assert np.all(np.abs(got - _exact_gram(A, B)) <= _gram_bound(A, B))
    G64 = torch.full((q, p), np.nan, dtype=torch.float64, device="cuda")
    ctx.gram(dA, p, dB, q, nrows, G64)
    ref64 = host(G64).T
    scale = np.outer(np.linalg.norm(A, axis=1), np.linalg.norm(B, axis=1))
    assert np.all(np.abs(got - ref64) <= 1e-14 * scale)
    G2 = torch.full((q, p), np.nan, dtype=torch.float64, device="cuda")
    ctx.gram(dA, p, dB, q, nrows, G2, dtype=tps.F64_TC)
    torch.cuda.synchronize()
    assert torch.equal(G, G2)


@pytest.mark.parametrize("nrows,p,q", [(131584, 40, 8), (100001, 8, 8), (5003, 33, 4)])
def test_gram_tc_graded(ctx, nrows, p, q):
    # columns spanning many binades (1e-8 .. 1e8), rows inside a column over 1e-12 .. 1e12
    # (so one 64-row block's scale differs from the next), entries over 1e-6 .. 1, zeros
    from paper_2111_02534_gb300 import tps
    rng = np.random.default_rng(nrows + p)
    A = rng.standard_normal((p, nrows)) * 10.0 ** rng.uniform(-6, 0, (p, nrows))
    A *= 10.0 ** rng.uniform(-12, 12, nrows)[None, :] * 10.0 ** rng.uniform(-8, 8, p)[:, None]
    B = rng.standard_normal((q, nrows)) * 10.0 ** rng.uniform(-12, 12, nrows)[None, :]
    A[:, ::97] = 0.0
    B[:, 5] = 0.0
    G = torch.full((q, p), np.nan, dtype=torch.float64, device="cuda")
    ctx.gram(dev(A), p, dev(B), q, nrows, G, dtype=tps.F64_TC)
    got = host(G).T
    assert np.all(np.abs(got - _exact_gram(A, B)) <= _gram_bound(A, B) + 1e-300)


def test_gram_tc_rejects_wide_blocks(ctx):
    from paper_2111_02534_gb300 import tps
    x = dev(random_block(9, 100, 1))
    G = torch.empty(81, dtype=torch.float64, device="cuda")
    with pytest.raises(tps.TpsError):
        ctx.gram(x, 9, x, 9, 100, G, dtype=tps.F64_TC)
    y = dev(random_block(65, 100, 1))
    G = torch.empty(65, dtype=torch.float64, device="cuda")
    with pytest.raises(tps.TpsError):
        ctx.gram(y, 65, x, 1, 100, G, dtype=tps.F64_TC)


@pytest.mark.parametrize("nrows,p,q,beta", [(131584, 24, 8, 0.0), (100003, 70, 3, 1.0),
                                            (513, 1, 17, -0.5), (1000, 0, 4, 2.0),
                                            # column tiles 1, 2, 4 (ragged), 8, 8 + 1
                                            (40001, 11, 1, 1.0), (3001, 5, 2, 0.0),
                                            (131584, 32, 5, -1.0), (20003, 9, 9, 0.5),
                                            # staged split path: partial last tile, p in
                                            # two slabs, two column groups
                                            (131590, 36, 8, 1.0), (200002, 100, 12, -1.0),
                                            # two and three column groups per CTA, four
                                            # (two CTA groups), ragged q
                                            (131584, 40, 24, 0.0), (131590, 33, 16, 1.0),
                                            (150000, 64, 20, -1.0), (140000, 17, 32, 0.5)])
@pytest.mark.parametrize("dtype", ["f64", "f64_tc"])
def test_block_update(ctx, nrows, p, q, beta, dtype):
    from paper_2111_02534_gb300 import tps
    dt = tps.F64_TC if dtype == "f64_tc" else tps.F64
    A = random_block(max(p, 1), nrows, 3)[:p]
    Y = np.random.default_rng(4).standard_normal((p, q))
    C0 = random_block(q, nrows, 5)
    Cd = dev(C0)
    if p > 64:
        with pytest.raises(tps.TpsError):
            ctx.block_update(dev(A), p, dev(Y.T.copy()), q, beta, Cd, nrows, dtype=dt)
        return
    ctx.block_update(dev(A) if p else None, p, dev(Y.T.copy()) if p else None, q, beta, Cd, nrows,
                     ldy=max(p, 1), dtype=dt)
    ref = beta * C0 + (Y.T @ A if p else 0.0)
    assert np.max(np.abs(host(Cd) - ref)) <= 1e-13 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("nrows,p,q", [(70001, 48, 8), (4099, 64, 13), (1000, 17, 3),
                                       # even row counts: A streamed through shared memory
                                       # by bulk copies (partial last tile, last k tile of
                                       # 4 and of 8 indices, two column groups)
                                       (131590, 36, 8), (262144, 64, 8), (100002, 40, 16),
                                       (64, 9, 2)])
def test_block_update_tc_graded(ctx, nrows, p, q):
    # digit-split update on data spanning many binades: rows scaled over 1e-12 .. 1e12,
    # entries within a row over 1e-6 .. 1, Y columns over 1e-8 .. 1e8, exact zeros; the
    # bound per entry is the scheme's, 2^-53 max_k |A[r][k]| sum_k |Y[k][j]| (with slack 4),
    # plus the worst-case rounding of the FP64 reference, p 2^-53 sum_k |Y[k][j] A[r][k]|
    from paper_2111_02534_gb300 import tps
    rng = np.random.default_rng(nrows)
    A = rng.standard_normal((p, nrows)) * 10.0 ** rng.uniform(-6, 0, (p, nrows))
    A *= 10.0 ** rng.uniform(-12, 12, nrows)[None, :]
    A[:, ::97] = 0.0
    Y = rng.standard_normal((p, q)) * 10.0 ** rng.uniform(-8, 8, q)[None, :]
    Cd = dev(np.zeros((q, nrows)))
    ctx.block_update(dev(A), p, dev(Y.T.copy()), q, 0.0, Cd, nrows, ldy=p, dtype=tps.F64_TC)
    got = host(Cd)
    ref = Y.T @ A
    bound = 4 * 2.0 ** -53 * np.outer(np.abs(Y).sum(axis=0), np.abs(A).max(axis=0))
    bound += p * 2.0 ** -53 * (np.abs(Y).T @ np.abs(A))
    assert np.all(np.abs(got - ref) <= bound + 1e-300)
    assert np.all(got[:, ::97] == 0.0)


@pytest.mark.parametrize("m,kind", [(1, "rand"), (2, "rand"), (7, "rand"), (32, "rand"),
                                    (64, "rand"), (40, "cluster"), (33, "graded"),
                                    (64, "graded"), (16, "jdlike"), (24, "jdlike"),
                                    (32, "jdlike"), (32, "degenerate"), (20, "equal"),
                                    (9, "zero"), (48, "tiny_gaps")])
def test_small_eigh(ctx, m, kind):
    # the default eigensolver (FP32 Jacobi + FP64 refinement): random spectra, tight
    # clusters, graded magnitudes, the spectra of Jacobi-Davidson projections (a few close
    # low Ritz values under a wide spread), exactly repeated and all-equal eigenvalues
    rng = np.random.default_rng(m)
    if kind == "rand":
        A = rng.standard_normal((m, m))
        A = A + A.T
    elif kind == "zero":
        A = np.zeros((m, m))
    else:
        Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
        if kind == "cluster":
            d = np.repeat(np.array([-3.0, -1e-3, 0.0, 1e-12, 2.0]), m // 5 + 1)[:m] + 1e-14 * rng.standard_normal(m)
        elif kind == "graded":
            d = np.logspace(-12, 3, m) * np.where(np.arange(m) % 2, -1, 1)
        elif kind == "jdlike":
            d = np.concatenate([np.sort(rng.uniform(-0.02, 0.0, 8)), 10 ** rng.uniform(-1, 2.5, m - 8)])
        elif kind == "degenerate":
            d = np.concatenate([np.full(6, -0.01), np.full(4, -0.0099999), 10 ** rng.uniform(-1, 2.5, m - 10)])
        elif kind == "equal":
            d = np.full(m, 2.5)
        else:  # eigenvalues 1e-9 apart around 1, and a wide spread
            d = np.concatenate([1.0 + 1e-9 * np.arange(m // 2), 10 ** rng.uniform(-2, 2, m - m // 2)])
        A = (Q * d) @ Q.T
        A = 0.5 * (A + A.T)
    th = torch.empty(m, dtype=torch.float64, device="cuda")
    Y = torch.empty(m, m, dtype=torch.float64, device="cuda")
    ctx.small_eigh(dev(A.T.copy()), m, th, Y)
    w, Yh = host(th), host(Y).T          # Y is column-major
    ref = np.linalg.eigvalsh(A)
    nrm = np.linalg.norm(A, 2)
    nrm = max(nrm, 1e-300)
    assert np.all(np.diff(w) >= 0)
    assert np.max(np.abs(w - ref)) <= 1e-14 * nrm * m
    assert np.max(np.abs(Yh.T @ Yh - np.eye(m))) <= 1e-13 * m
    assert np.max(np.abs(A @ Yh - Yh * w)) <= 1e-14 * nrm * m


def test_orthonormalize(ctx):
    nrows = 50000
    rng = np.random.default_rng(9)
    Q, _ = np.linalg.qr(rng.standard_normal((nrows, 6)))
    T = rng.standard_normal((nrows, 5))
    T[:, 3] = 2 * T[:, 0] - T[:, 1] + 1e-12 * rng.standard_normal(nrows)  # dependent column
    T[:, 4] = Q[:, 2] * 3.0                                                # inside span(Q)
    Td = dev(T.T.copy())
    rank = ctx.orthonormalize(dev(Q.T.copy()), 6, Td, 5, nrows)
    assert rank == 3
    Z = host(Td)[:rank].T
    assert np.max(np.abs(Z.T @ Z - np.eye(rank))) <= 1e-13
    assert np.max(np.abs(Q.T @ Z)) <= 1e-13
    ref = blocks.orthonormal_complement_step(Q, T[:, :3])
    # same subspace as the Householder definition
    assert np.linalg.norm(ref @ (ref.T @ Z) - Z) <= 1e-10


@pytest.mark.parametrize("use_prec", [1, 0])
def test_correction_converged_krylov_is_exact(use_prec):
    # 20 steps on a 34-dimensional complement: the GMRES residual is at rounding level
    # (about 1e-15 for this case), so the iterate is the exact solution of Eq. jdcor
    require_gpu()
    n = (6, 6)
    P = problem_1d(20.0, 1.0, 1.0, n, (3.0, 3.0), 1.0, 1.0)
    c = make_ctx_1d(20.0, 1.0, n, (3.0, 3.0), 1.0, 1.0)
    H = P.assemble_dense()
    w, U = np.linalg.eigh(H)
    rng = np.random.default_rng(1)
    X = U[:, :2] + 1e-2 * rng.standard_normal((P.N, 2))
    Qt, _ = np.linalg.qr(X)
    th = np.array([Qt[:, i] @ H @ Qt[:, i] for i in range(2)])
    R = H @ Qt - Qt * th
    R = R - Qt @ (Qt.T @ R)
    T = torch.empty(2, P.N, dtype=torch.float64, device="cuda")
    c.correction(dev(Qt.T.copy()), 2, dev(R.T.copy()), dev(th), 2, 20 if use_prec else 34,
                 use_prec, -0.7, T)
    got = host(T)
    for i in range(2):
        ref = blocks.correction_exact(H, Qt, th[i], R[:, i])
        assert np.linalg.norm(got[i] - ref) <= 1e-8 * np.linalg.norm(ref)


def test_correction_matches_textbook_gmres():
    # a few steps: same Krylov space and minimisation as the oracle's textbook GMRES
    require_gpu()
    n = (10, 8)
    L = (4.0, 4.0)
    P = problem_1d(20.0, 1.0, 1.0, n, L, 1.0, 1.0)
    c = make_ctx_1d(20.0, 1.0, n, L, 1.0, 1.0)
    H = P.assemble_dense()
    w, U = np.linalg.eigh(H)
    rng = np.random.default_rng(2)
    Qt, _ = np.linalg.qr(U[:, :3] + 1e-2 * rng.standard_normal((P.N, 3)))
    th = np.array([Qt[:, i] @ H @ Qt[:, i] for i in range(3)])
    R = H @ Qt - Qt * th
    shift, steps = -0.9, 6
    T = torch.empty(3, P.N, dtype=torch.float64, device="cuda")
    c.correction(dev(Qt.T.copy()), 3, dev(R.T.copy()), dev(th), 3, steps, 1, shift, T)
    got = host(T)
    Kinv = lambda Y: apply_dense(P, np.asarray(Y).T, shift).T
    Pm = np.eye(P.N) - Qt @ Qt.T
    for i in range(3):
        A = lambda v: blocks.projected_preconditioner(Kinv, Qt, Pm @ ((H - th[i] * np.eye(P.N)) @ (Pm @ v)))
        b = -blocks.projected_preconditioner(Kinv, Qt, R[:, i])
        x, _ = blocks.gmres(A, b, steps)
        assert np.linalg.norm(got[i] - x) <= 1e-9 * np.linalg.norm(x)
        assert abs(Qt.T @ got[i]).max() <= 1e-10 * np.linalg.norm(got[i])
