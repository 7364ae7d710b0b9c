"""Seeded synthetic workloads for the three-body tensor-product eigensolver.

This module holds only workload parameters and seeded random arrays.  It
contains none of the method's arithmetic (no grids, no potentials, no
operators): both the CUDA path and the independent CPU oracle read their
inputs from here and compute everything else on their own.

Workloads (physical masses, hbar = 1, heavy-heavy-light system of Sec. 2):

* ``1d_n64``   -- 1D, M = 20, m = 1, n = 64 per Jacobi coordinate on the
  periodic box [-20, 20), Gaussian heavy-light well v0 = 1, sigma = 1,
  4 lowest states that are even under heavy-particle exchange.
* ``1d_n512``  -- the same 1D system at n = 512 per coordinate, M/m = 40,
  v0 tuned so that the heavy-light pair is bound by E0 = 1e-3, 8 lowest
  exchange-even states, block size 8.
* ``2d_n48``   -- 2D, n = 48 per Cartesian Jacobi component (5.3 M
  unknowns), M/m = 20, v0 = 2, sigma = 1, 4 lowest states, block size 8.
* ``sweep``    -- 256 independent 1D instances drawn with PCG64(seed=3):
  M/m ~ U[1, 40], heavy-light binding E0 ~ logU[1e-4, 1], sigma uniform in
  {0.5, 1, 2}, n uniform in {128, 192, 256, 384}, L = 20, 4 states each.
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Tuple

import numpy as np

GAUSS = 0
LORENTZ3 = 1

ANY = 0
X_EVEN = 1
X_ODD = 2


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    dim: int
    M: float
    m: float
    hbar: float
    n: Tuple[int, ...]          # grid points per coordinate: (x, y) or (x1, x2, y1, y2)
    L: Tuple[float, ...]        # half box length per coordinate
    shape: int
    sigma: float
    v0: Optional[float]         # well depth, or None when tuned from E0
    E0: Optional[float]         # heavy-light binding energy (> 0) used to tune v0
    parity: int
    k: int
    block: int

    @property
    def N(self) -> int:
        return int(np.prod(self.n))


WORKLOADS = {
    "1d_n64": Workload("1d_n64", 1, 20.0, 1.0, 1.0, (64, 64), (20.0, 20.0),
                       GAUSS, 1.0, 1.0, None, X_EVEN, 4, 4),
    "1d_n512": Workload("1d_n512", 1, 40.0, 1.0, 1.0, (512, 512), (20.0, 20.0),
                        GAUSS, 1.0, None, 1e-3, X_EVEN, 8, 8),
    "2d_n48": Workload("2d_n48", 2, 20.0, 1.0, 1.0, (48, 48, 48, 48),
                       (20.0, 20.0, 20.0, 20.0), GAUSS, 1.0, 2.0, None, ANY, 4, 8),
}


def random_block(nvec: int, N: int, seed: int) -> np.ndarray:
    """nvec wave-function vectors with entries uniform in [-1, 1), FP64, shape [nvec, N]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(nvec, N))


def random_normal_block(nvec: int, N: int, seed: int) -> np.ndarray:
    """nvec vectors with standard-normal entries, FP64, shape [nvec, N]."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=(nvec, N))


def sweep_instances(count: int = 256, seed: int = 3):
    """Parameters of the batched 1D sweep: a list of dicts (M, m, E0, sigma, n, L)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        ratio = rng.uniform(1.0, 40.0)
        E0 = float(np.exp(rng.uniform(np.log(1e-4), np.log(1.0))))
        sigma = float(rng.choice([0.5, 1.0, 2.0]))
        n = int(rng.choice([128, 192, 256, 384]))
        out.append(dict(M=float(ratio), m=1.0, E0=E0, sigma=sigma, n=n, L=20.0))
    return out


def warmstart_instances(count: int, seed: int, ratio=(1.0, 40.0), E0=(1e-4, 1.0),
                        sigmas=(0.5, 1.0, 2.0), ns=(128, 192, 256, 384), L: float = 20.0,
                        dim: int = 1):
    """Parameters of instances for the learned warm start (same fields as sweep_instances,
    plus dim): M/m uniform in `ratio`, E0 log-uniform in `E0`, sigma and n drawn from the
    given sets; n points and half-width L on every Cartesian component."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        r = rng.uniform(*ratio)
        e = float(np.exp(rng.uniform(np.log(E0[0]), np.log(E0[1]))))
        s = float(rng.choice(list(sigmas)))
        n = int(rng.choice(list(ns)))
        out.append(dict(M=float(r), m=1.0, E0=e, sigma=s, n=n, L=L, dim=dim))
    return out
