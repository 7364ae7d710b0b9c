"""Helpers shared by the GPU parity tests: build matching CUDA contexts and oracle problems
from the same workload parameters (each side computes its own grid, D2 and potential)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def make_ctx_1d(M, m, n, L, v0, sigma, shape=0, alpha=None, V=None):
    from paper_2111_02534_gb300 import tps
    ctx = tps.Context(1, 0)
    if alpha is not None:
        ctx.set_alpha(alpha)
    else:
        ctx.set_masses(M, m, 1.0)
    ctx.set_grid(list(n), list(L))
    if V is not None:
        ctx.set_potential(np.ascontiguousarray(V, dtype=np.float64).ravel())
    else:
        ctx.set_pair_potential(shape, v0, sigma)
    return ctx


def make_ctx_2d(M, m, n, L, v0, sigma, shape=0):
    from paper_2111_02534_gb300 import tps
    ctx = tps.Context(2, 0)
    ctx.set_masses(M, m, 1.0)
    ctx.set_grid(list(n), list(L))
    ctx.set_pair_potential(shape, v0, sigma)
    return ctx


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()
