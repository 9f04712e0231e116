"""CPU pin of the large-subspace Rayleigh-Ritz scheme (m up to 512, Section 4.2.2's dense
shapes): FP32 eigenvectors of the projected matrix T, made orthogonal in FP64 by two
Newton-Schulz steps Q <- Q (3 I - Q^T Q) / 2 (Higham, "Functions of Matrices", 8.3), then an
FP64 eigendecomposition of Q^T T Q, give T's eigenpairs to FP64 accuracy.

The algebra checked: with E = Q^T Q - I, one step gives Q'^T Q' - I = -3/4 E^2 + 1/4 E^3, so an
FP32-level E (1e-6 .. 1e-5) falls to FP64 rounding in two steps but not in one.  numpy's FP32
eigh stands in for the FP32 Jacobi sweeps and FP64 eigh for the FP64 sweeps; the FP32 vectors are
perturbed to the orthogonality a product of FP32 rotations reaches at m = 512.
"""
import numpy as np
import pytest


def _problem(m, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((m, m))
    w, V = np.linalg.eigh((G + G.T) / 2)
    w[:24] = 5.0 + 1e-4 * w[:24]                       # a tight cluster, as in the solver's stalls
    T = (V * w) @ V.T
    return (T + T.T) / 2, rng


def _fp32_vectors(T, rng, level):
    _, Q32 = np.linalg.eigh(T.astype(np.float32))
    Q = Q32.astype(np.float64)
    Q += level * rng.standard_normal(Q.shape) / np.sqrt(Q.shape[0])
    return Q


def _newton_schulz(Q, steps):
    I = np.eye(Q.shape[1])
    for _ in range(steps):
        Q = Q @ (3 * I - Q.T @ Q) / 2
    return Q


def _orth(Q):
    return np.abs(Q.T @ Q - np.eye(Q.shape[1])).max()


def test_one_step_identity():
    """Q'^T Q' - I = -3/4 E^2 + 1/4 E^3 for Q' = Q (3 I - Q^T Q) / 2 (exact algebra, FP64)."""
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    Q = Q + 1e-3 * rng.standard_normal(Q.shape)
    E = Q.T @ Q - np.eye(40)
    Q1 = _newton_schulz(Q, 1)
    assert np.allclose(Q1.T @ Q1 - np.eye(40), -0.75 * E @ E + 0.25 * E @ E @ E, rtol=0, atol=1e-14)


@pytest.mark.parametrize("m", [192, 512])
def test_two_steps_reach_fp64_eigenpairs(m):
    T, rng = _problem(m, m)
    Q0 = _fp32_vectors(T, rng, 1e-5)
    assert 1e-6 < _orth(Q0) < 1e-4                     # FP32-level orthogonality to start from
    ref = np.linalg.eigvalsh(T)
    scale = np.abs(ref).max()
    Q = _newton_schulz(Q0, 2)
    assert _orth(Q) <= 1e-14
    A = Q.T @ T @ Q
    theta, Y = np.linalg.eigh((A + A.T) / 2)
    X = Q @ Y
    assert np.abs(np.sort(theta) - ref).max() <= 1e-13 * scale
    assert np.abs(T @ X - X * theta).max() <= 1e-13 * scale
    assert _orth(X) <= 1e-13


def test_one_step_is_not_enough():
    """From the same start, one step leaves ~E^2 ~ 1e-10: the eigenvalues of Q^T T Q are then off
    by far more than FP64 rounding, so the second step is needed."""
    T, rng = _problem(512, 512)
    Q0 = _fp32_vectors(T, rng, 1e-5)
    Q = _newton_schulz(Q0, 1)
    assert _orth(Q) > 1e-12
    theta = np.linalg.eigvalsh(Q.T @ T @ Q)
    assert np.abs(theta - np.linalg.eigvalsh(T)).max() > 1e-12 * np.abs(theta).max()
