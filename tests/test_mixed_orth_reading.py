"""CPU pin of the solver's mixed-arithmetic re-orthogonalisation of an FP64 subspace (block
CGS2 + CholeskyQR2, Section 3.1 step (1)), restated in numpy: the first pass's Gram G1 = V^T W
is taken in FP32 arithmetic and only steers; W is updated in FP64 with whatever G1 is; the
second pass's Gram G2 and W1^T W1 are FP64; its correction V C (C = -G2 R1^-1, small after the
first pass) and the CholeskyQR second pass's W2 (R2^-1 - I) are formed in FP32 arithmetic when
their coefficients are at most 1e-5; the coefficients recorded are G1 + G2 and R2 R1.

Checked on a hard step (W mostly inside span(V), remainder 1e-3 of it): the result is
orthonormal to FP64 rounding, orthogonal to V and consistent (W = V G + Q R) within the FP32
correction's stated scale 2^-23 * 1e-5, and agrees with the all-FP64 oracle
(oracle.bks.orth_block) to that scale; with one pass only it is not (the second pass is what
makes an FP32-steered first pass safe).
"""
import numpy as np
import pytest

from oracle import bks

F32, F64 = np.float32, np.float64


def _trunc32(x):
    """FP64 -> FP32 by truncating the significand (the kernels' integer conversion): the 29 low
    fraction bits are cleared, after which the value is exact in FP32."""
    bits = np.ascontiguousarray(x, dtype=F64).view(np.uint64) & ~np.uint64((1 << 29) - 1)
    return bits.view(F64).astype(F32)


def _chol_upper(M):
    return np.linalg.cholesky(M).T                        # M = R^T R, R upper triangular


def mixed_orth(V, W, two_passes=True):
    G1 = (V.astype(F32).T @ W.astype(F32)).astype(F64)     # FP32 arithmetic, steering only
    W1 = W - V @ G1                                        # FP64 update
    if not two_passes:
        R = _chol_upper(W1.T @ W1)
        return G1, W1 @ np.linalg.inv(R), R
    G2 = V.T @ W1                                          # FP64 Gram of the same sweep
    R1 = _chol_upper(W1.T @ W1)
    R1i = np.linalg.inv(R1)
    C = -G2 @ R1i
    assert np.abs(C).max() <= 1e-5                         # the FP32 correction's condition
    VC = (_trunc32(V) @ C.astype(F32)).astype(F64)         # correction in FP32 arithmetic
    W2 = W1 @ R1i + VC
    R2 = _chol_upper(W2.T @ W2)
    D = np.linalg.inv(R2) - np.eye(R2.shape[0])
    assert np.abs(D).max() <= 1e-5
    Q = W2 + (_trunc32(W2) @ D.astype(F32)).astype(F64)    # W2 R2^-1, correction in FP32
    return G1 + G2, Q, R2 @ R1


def _step(seed, n=20000, k=32, b=4, rem=1e-3):
    rng = np.random.default_rng(seed)
    V, _ = np.linalg.qr(rng.standard_normal((n, k)))
    W = V @ rng.standard_normal((k, b)) + rem * rng.standard_normal((n, b))
    return V, W


@pytest.mark.parametrize("seed", [1, 2])
def test_mixed_arithmetic_matches_all_fp64(seed):
    V, W = _step(seed)
    G, Q, R = mixed_orth(V, W)
    # the FP32 correction's rounding (V truncated to FP32, times |C| <= 1e-5) stays below
    # 2^-23 * 1e-5 ~ 1.2e-12 of the unit columns' scale; the all-FP64 step sits at ~1e-17 here
    fp32_scale = 2.0 ** -23 * 1e-5
    assert np.abs(V.T @ Q).max() <= fp32_scale             # orthogonal to the basis
    assert np.abs(Q.T @ Q - np.eye(Q.shape[1])).max() <= 1e-14
    assert np.abs(W - V @ G - Q @ R).max() <= fp32_scale * np.abs(W).max()
    state = {"counter": 0, "replacements": 0}
    Qo, Go, Ro = bks.orth_block(V, W, 1.0, 1, state)
    assert state["replacements"] == 0
    assert np.abs(Q - Qo).max() <= fp32_scale              # the same block, both ways
    assert np.abs(R - Ro).max() <= 1e-13 * np.abs(W).max()
    assert np.abs(G - Go).max() <= 1e-13 * np.abs(W).max()


def test_one_fp32_steered_pass_is_not_enough():
    V, W = _step(3)
    _, Q, _ = mixed_orth(V, W, two_passes=False)
    assert np.abs(V.T @ Q).max() > 1e-6                    # FP32 steering error, not removed
