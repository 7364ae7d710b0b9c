"""Pins for oracle.two_body: Table 1 (1D) v0 values to the printed 8 digits."""
import json
import os

import numpy as np
import pytest

from oracle.two_body import tune_v0, two_body_energy
from oracle.hamiltonian import GAUSS, LORENTZ3

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _table1():
    with open(os.path.join(GOLD, "table1.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("row", [0, 1, 2])
def test_table1_v0(row):
    r = _table1()["rows"][row]
    # box large enough that exp(-sqrt(2 E0) L) is negligible; h ~ 0.2-0.4 resolves f_G
    L, n = {0: (100.0, 512), 1: (100.0, 512), 2: (200.0, 1024)}[row]
    v0 = tune_v0(r["E0"], 1.0, 1.0, GAUSS, n, L)
    assert abs(v0 - r["v0"]) <= 0.5e-8 + 1e-10


@pytest.mark.parametrize("E0,shape", [(0.1, GAUSS), (0.01, LORENTZ3), (0.5, GAUSS)])
def test_tuned_depth_gives_binding_energy(E0, shape):
    v0 = tune_v0(E0, 0.8, 1.3, shape, 256, 40.0)
    assert two_body_energy(v0, 0.8, 1.3, shape, 256, 40.0) == pytest.approx(-E0, rel=1e-11)


def test_mass_and_width_scaling():
    # -1/(2 mu) d2 - v0 f(x/s): scaling x = s u gives depth v0(mu, s, E0) = v0(1, 1, E0 mu s^2)/(mu s^2)
    mu, s, E0 = 0.7, 2.0, 0.05
    a = tune_v0(E0, mu, s, GAUSS, 512, 80.0)
    b = tune_v0(E0 * mu * s * s, 1.0, 1.0, GAUSS, 512, 40.0) / (mu * s * s)
    assert a == pytest.approx(b, rel=1e-9)


def _table3():
    with open(os.path.join(GOLD, "table3_v0.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("shape,key,L,n,tol", [
    (GAUSS, "gauss", 30.0, 192, 1.0e-8),
    # f_L has poles at xi = +-i, so its spectral error is ~exp(-pi/h): needs h = 0.15
    (LORENTZ3, "lorentz3", 30.0, 400, 2.0e-8),
])
def test_table3_v0_2d(shape, key, L, n, tol):
    from oracle.two_body import tune_v0_2d_iterative
    row = _table3()["rows"][0]
    v0 = tune_v0_2d_iterative(row["E0"], 1.0, 1.0, shape, n, L)
    assert abs(v0 - row[key]) <= tol


def test_2d_dense_and_iterative_agree():
    from oracle.two_body import tune_v0_2d_iterative
    a = tune_v0(0.2, 1.0, 1.0, GAUSS, 24, 8.0, dim=2)
    b = tune_v0_2d_iterative(0.2, 1.0, 1.0, GAUSS, 24, 8.0)
    assert a == pytest.approx(b, rel=1e-11)


def _v0_rayleigh_long_double(v0, E0, mu, sigma, n, L):
    """v0 as the Rayleigh quotient psi^T (T + E0) psi / psi^T F psi of the pencil, in
    extended precision, with T from the closed-form D2 entries and psi the FP64 ground
    state of T - v0 F.  The quotient is stationary at the eigenvector, so an FP64 psi
    gives v0 to extended-precision rounding."""
    ld = np.longdouble
    pi = 4 * np.arctan(ld(1))          # pi to extended precision (np.pi is FP64)
    x = -ld(L) + np.arange(n, dtype=ld) * (2 * ld(L) / n)
    h = 2 * pi / n
    d = np.subtract.outer(np.arange(n), np.arange(n))
    with np.errstate(divide="ignore"):
        D = -np.where(d % 2 == 0, ld(1), ld(-1)) / (2 * np.sin(d.astype(ld) * h / 2) ** 2)
    D[np.arange(n), np.arange(n)] = -ld(n) ** 2 / 12 - ld(1) / 6     # -pi^2/(3h^2) - 1/6
    T = -D * (pi / ld(L)) ** 2 / (2 * ld(mu))
    f = np.exp(-(np.abs(x) / ld(sigma)) ** 2)
    w, V = np.linalg.eigh(T.astype(np.float64) - v0 * np.diag(f.astype(np.float64)))
    psi = V[:, 0].astype(ld)
    return float((psi @ (T @ psi) + ld(E0) * (psi @ psi)) / (psi @ (f * psi)))


@pytest.mark.parametrize("E0,mu,sigma,n", [(1e-4, 0.95, 2.0, 128), (3e-4, 0.97, 0.5, 192),
                                           (0.3, 0.8, 1.0, 128)])
def test_v0_small_binding_extended_precision(E0, mu, sigma, n):
    # near threshold T + E0 is ill-conditioned (cond ~ 1e6); v0 must still be accurate to
    # the FP64 representation of the grid operators (~2e-14 observed), which a
    # Cholesky-based generalized eigensolver does not reach (1e-11 .. 1e-10 observed)
    v0 = tune_v0(E0, mu, sigma, GAUSS, n, 20.0)
    ref = _v0_rayleigh_long_double(v0, E0, mu, sigma, n, 20.0)
    assert abs(v0 - ref) <= 1e-13 * ref
