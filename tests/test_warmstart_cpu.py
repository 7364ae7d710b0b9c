"""Host logic of the warm-start driver: the canonical form of degenerate 2D targets."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_canonical_targets_undo_a_rotation_of_a_degenerate_pair():
    from paper_2111_02534_gb300 import warmstart
    q = 4
    px = py = q * q
    s1 = np.array([1.0, 1.0, -1.0, 1.0])           # modes 1, cos, sin, cos 2
    sign = np.outer(np.repeat(s1, q), np.repeat(s1, q))
    rng = np.random.Generator(np.random.PCG64(5))
    A = rng.normal(size=(px, py))
    even, odd = A * (sign > 0), A * (sign < 0)        # eigenvectors of the reflection
    c, s = np.cos(0.7), np.sin(0.7)
    other = rng.normal(size=(px, py))
    T = np.stack([other, c * even + s * odd, -s * even + c * odd])
    lam = np.array([-2.0, -1.0, -1.0 + 1e-13])        # the last two degenerate
    out = warmstart.canonical_targets(torch.from_numpy(T.astype(np.float32)), lam, px, py)
    out = out.numpy().astype(np.float64)
    assert np.allclose(out[0], T[0], atol=1e-6)       # a simple eigenvalue is untouched

    def cos2(a, b):
        return (a * b).sum() ** 2 / ((a * a).sum() * (b * b).sum())
    assert cos2(out[1], even) > 1 - 1e-10             # even under the reflection first
    assert cos2(out[2], odd) > 1 - 1e-10
