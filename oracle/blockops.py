"""Table 1 dense operations on tall-and-skinny blocks, FP64 numpy.  Test infrastructure only.

AA, BB, CC are n x b tall blocks; A, B small matrices; alpha, beta scalars (Table 1).
"""
from __future__ import annotations

import numpy as np


def mv_times_mat_add_mv(alpha, AA, B, beta, CC):
    """MvTimesMatAddMv ("op1"): CC <- alpha * AA @ B + beta * CC."""
    return alpha * (AA @ B) + beta * CC


def mv_trans_mv(alpha, AA, BB):
    """MvTransMv ("op3"): A <- alpha * AA^T @ BB."""
    return alpha * (AA.T @ BB)


def mv_scale1(alpha, AA):
    """MvScale1: BB <- alpha * AA."""
    return alpha * AA


def mv_scale2(AA, vec):
    """MvScale2: BB <- AA @ diag(vec)."""
    return AA * np.asarray(vec)[None, :]


def mv_add_mv(alpha, AA, beta, BB):
    """MvAddMv: CC <- alpha * AA + beta * BB."""
    return alpha * AA + beta * BB


def mv_dot(AA, BB):
    """MvDot: vec[i] <- AA[:, i]^T BB[:, i]."""
    return np.einsum("ij,ij->j", AA, BB)


def mv_norm(AA):
    """MvNorm: column 2-norms."""
    return np.sqrt(np.einsum("ij,ij->j", AA, AA))


def chol_upper(S: np.ndarray, rel_pivot: float, abs_pivot: float):
    """Upper-triangular R with R^T R = S (Cholesky, column by column).

    Returns (R, ok).  ok is False when a pivot d_j (the squared diagonal) is not positive,
    when sqrt(d_j) < rel_pivot * sqrt(S_jj) (column j nearly dependent on the earlier
    columns) or when sqrt(d_j) <= abs_pivot (column j numerically zero).
    """
    b = S.shape[0]
    R = np.zeros((b, b))
    for j in range(b):
        for i in range(j):
            R[i, j] = (S[i, j] - R[:i, i] @ R[:i, j]) / R[i, i]
        d = S[j, j] - R[:j, j] @ R[:j, j]
        if not (d > 0.0) or np.sqrt(d) < rel_pivot * np.sqrt(S[j, j]) or np.sqrt(d) <= abs_pivot:
            return R, False
        R[j, j] = np.sqrt(d)
    return R, True


def cholqr(W: np.ndarray, rel_pivot: float, abs_pivot: float):
    """One Cholesky-QR pass: S = W^T W = R^T R, Q = W R^{-1}.  Returns (Q, R, ok)."""
    S = W.T @ W
    R, ok = chol_upper(S, rel_pivot, abs_pivot)
    if not ok:
        return W, R, False
    Q = np.linalg.solve(R.T, W.T).T
    return Q, R, True


def cholqr2(W: np.ndarray, rel_pivot: float, abs_pivot: float):
    """CholeskyQR2 (Fukaya et al. 2014): two Cholesky-QR passes, R = R2 R1."""
    Q1, R1, ok = cholqr(W, rel_pivot, abs_pivot)
    if not ok:
        return W, R1, False
    Q, R2, ok = cholqr(Q1, rel_pivot, 0.0)
    if not ok:
        return W, R2, False
    return Q, R2 @ R1, True
