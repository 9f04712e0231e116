"""Singular values of a directed graph's adjacency matrix, FP64 numpy.  Test infrastructure only.

The paper's billion-node page graph is directed, so its adjacency matrix A is not symmetric
and the paper computes a singular value decomposition of A instead of an eigendecomposition
(Section 4.3.2), with the same Block Krylov-Schur solver.  The paper does not say how the
solver is applied; this follows the standard reduction (Golub & Van Loan Section 8.6.1):

  * the eigenpairs (theta_i, v_i) of the symmetric positive semidefinite A^T A are found by
    the Block Krylov-Schur iteration of bks.py, with the operator X -> A^T (A X) in place of
    the SpMM (two SpMMs per block: A X, then A^T applied to the result), largest first;
  * sigma_i = sqrt(theta_i) are the singular values and v_i the right singular vectors;
  * the left singular vectors are u_i = A v_i / sigma_i (u_i = 0 when sigma_i = 0).

A^T is the transposed pattern: the non-zero (i, j) of A becomes (j, i).  The convergence test is
bks.py's, applied to the eigenpairs of A^T A (rho_i <= tol * max(theta_i, 1e-3 max theta)).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import bks, core


def transpose(rowptr: np.ndarray, colidx: np.ndarray):
    """CSR pattern of A^T: entry (i, j) of A becomes (j, i); column indices sorted."""
    n = rowptr.shape[0] - 1
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    cols = colidx.astype(np.int64)
    order = np.lexsort((rows, cols))            # by new row (= old column), then new column
    t_colidx = rows[order].astype(np.int32)
    counts = np.bincount(cols, minlength=n)
    t_rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=t_rowptr[1:])
    return t_rowptr, t_colidx


@dataclasses.dataclass
class SvdResult:
    svals: np.ndarray         # nsv singular values, descending
    right: np.ndarray         # n x nsv right singular vectors (largest-|entry| positive)
    left: np.ndarray          # n x nsv left singular vectors, A v_i / sigma_i
    eig: bks.Result           # the Krylov-Schur run on A^T A


def svds(rowptr, colidx, nsv: int, block: int, nblocks: int, tol: float, seed: int = 1,
         start=None, max_restarts: int = 500) -> SvdResult:
    """The nsv largest singular triplets of the 0/1 matrix (rowptr, colidx)."""
    t_rowptr, t_colidx = transpose(rowptr, colidx)

    def ata(X):
        return core.spmm(t_rowptr, t_colidx, core.spmm(rowptr, colidx, X))

    r = bks.block_krylov_schur(rowptr, colidx, nsv, block, nblocks, tol, "LA", start=start,
                               seed=seed, max_restarts=max_restarts, spmm=ata)
    sig = np.sqrt(np.maximum(r.evals, 0.0))
    V = r.evecs
    AV = core.spmm(rowptr, colidx, V)
    U = np.zeros_like(AV)
    pos = sig > 0.0
    U[:, pos] = AV[:, pos] / sig[pos]
    return SvdResult(sig, V, U, r)
