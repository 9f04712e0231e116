"""Block Krylov-Schur eigensolver, FP64 numpy.  Test infrastructure only.

The paper gives the generic projection iteration (Algorithm 1, Section 3.1): (1) update the
subspace S, (2) solve the projected problem S^T A S y = theta y, (3) form the residual
r = A x - x theta of the Ritz pair x = S y, (4) test convergence; with the block extension
(Section 3.1: block size b, NB blocks, subspace m = b * NB) that makes step (1) a sparse
matrix times dense block multiply (SpMM, Section 3.3) followed by re-orthogonalisation with
the Table 1 operations MvTransMv and MvTimesMatAddMv.  The solver is Anasazi's Block
Krylov-Schur (Section 1), which the paper cites but does not spell out; this follows Stewart's
Krylov-Schur decomposition A V_k = V_k S_k + V_res B^T, in block form:

  start   V_0 = CholQR2(start block)
  expand  for j = k/b .. NB-1:  W = A V_j;  block CGS2 against V_0..V_j (G = G1 + G2);
          CholQR2(W) = V_{j+1} R;  H[0:(j+1)b, jb:(j+1)b] = G,  H[(j+1)b:(j+2)b, jb:(j+1)b] = R
  project T = (H_m + H_m^T) / 2,  T = Y diag(theta) Y^T  (Jacobi), ordered by `which`
  test    rho_i = ||H[m:m+b, 0:m] y_i||  <=  tol * max(|theta_i|, 1e-3 * max|theta|)
          for the first nev; then the explicit residual ||A x_i - theta_i x_i|| must pass too
  restart keep k Ritz vectors: V_k <- V_m Y_k, residual block V_NB moves to slot k/b,
          H <- [diag(theta_k); B^T = H[m:m+b, :m] Y_k]

Readings where the paper is silent are listed in the module-level constants below.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import blockops, core, rng

# Readings (the paper is silent on these; the CUDA library makes the same choices):
REL_PIVOT = 1e-6        # CholQR pivot below 1e-6 * column norm -> column-wise fallback
ABS_BREAKDOWN = 1e-12   # remainder below 1e-12 * ||A||_est -> breakdown, random replacement
SMALL_THETA = 1e-3      # convergence scale floor, relative to the largest |theta|
STREAM_START = 4        # counter-RNG stream of the random start block
STREAM_REPLACE = 5      # counter-RNG stream of breakdown replacement vectors


@dataclasses.dataclass
class Result:
    evals: np.ndarray
    evecs: np.ndarray
    converged: bool
    nconv: int
    restarts: int
    spmm_blocks: int          # number of n x b block SpMMs
    ritz_resid: np.ndarray    # rho_i of the final Ritz pairs (first nev)
    resid: np.ndarray         # explicit ||A x_i - theta_i x_i||, first nev
    anorm: float
    replacements: int


def restart_size(nev: int, b: int, m: int) -> int:
    """Kept Ritz vectors at a restart: nev + (m - nev)//2, rounded down to a multiple of b,
    clamped to [ceil(nev/b)*b, m - b]."""
    k = nev + (m - nev) // 2
    k -= k % b
    lo = -(-nev // b) * b
    return max(lo, min(k, m - b))


def sort_order(theta: np.ndarray, which: str) -> np.ndarray:
    """LM: |theta| descending, ties -> larger theta first; LA: descending; SA: ascending."""
    if which == "LM":
        return np.lexsort((-theta, -np.abs(theta)))
    if which == "LA":
        return np.argsort(-theta, kind="stable")
    if which == "SA":
        return np.argsort(theta, kind="stable")
    raise ValueError(which)


def _random_direction(basis_list, n, seed, counter):
    """A unit vector orthogonal to every column of the given bases (two CGS passes)."""
    for attempt in range(8):
        r = rng.normal_block(n, 1, seed, STREAM_REPLACE, offset=(counter + attempt) * n)[:, 0]
        r0 = np.linalg.norm(r)
        for _ in range(2):
            for B in basis_list:
                if B.shape[1]:
                    r = r - B @ (B.T @ r)
        nr = np.linalg.norm(r)
        if nr > 1e-10 * r0:
            return r / nr, attempt + 1
    raise RuntimeError("could not draw a replacement direction (subspace fills R^n)")


def orth_block(Vb: np.ndarray, W: np.ndarray, anorm: float, seed: int, state: dict):
    """Block CGS2 of W against the orthonormal basis Vb, then CholQR2 of the remainder.

    Returns (Q, G, R) with W_in = Vb G + Q R, Q orthonormal and orthogonal to Vb.
    If CholQR2's pivot checks fail, falls back to column-wise two-pass Gram-Schmidt; a
    column whose remainder is below ABS_BREAKDOWN * anorm is replaced by a random direction
    and gets R[i, i] = 0 (breakdown: the Krylov space has become invariant there).
    """
    G1 = blockops.mv_trans_mv(1.0, Vb, W)
    W = blockops.mv_times_mat_add_mv(-1.0, Vb, G1, 1.0, W)
    G2 = blockops.mv_trans_mv(1.0, Vb, W)
    W = blockops.mv_times_mat_add_mv(-1.0, Vb, G2, 1.0, W)
    G = G1 + G2
    Q, R, ok = blockops.cholqr2(W, REL_PIVOT, ABS_BREAKDOWN * anorm)
    if ok:
        return Q, G, R
    n, b = W.shape
    Q = np.zeros((n, b))
    R = np.zeros((b, b))
    for i in range(b):
        w = W[:, i].copy()
        for _ in range(2):
            c = Vb.T @ w
            w -= Vb @ c
            G[:, i] += c
            d = Q[:, :i].T @ w
            w -= Q[:, :i] @ d
            R[:i, i] += d
        nr = np.linalg.norm(w)
        if nr > ABS_BREAKDOWN * anorm and nr > 0.0:
            Q[:, i] = w / nr
            R[i, i] = nr
        else:
            q, used = _random_direction([Vb, Q[:, :i]], n, seed, state["counter"])
            state["counter"] += used
            state["replacements"] += 1
            Q[:, i] = q
    return Q, G, R


def block_krylov_schur(rowptr, colidx, nev: int, block: int, nblocks: int, tol: float,
                       which: str = "LM", start=None, seed: int = 1, max_restarts: int = 500,
                       spmm=None) -> Result:
    """Eigenpairs of the 0/1 symmetric matrix A = (rowptr, colidx); see the module docstring."""
    n = rowptr.shape[0] - 1
    b = block
    m = b * nblocks
    if not (b >= 1 and nblocks >= 2 and 1 <= nev <= m - b and m + b <= n):
        raise ValueError("need 1 <= nev <= block*(nblocks-1) and block*(nblocks+1) <= n")
    if spmm is None:
        def spmm(X):
            return core.spmm(rowptr, colidx, X)
    if start is None:
        start = rng.normal_block(n, b, seed, STREAM_START)
    start = np.asarray(start, dtype=np.float64).reshape(n, b)

    V = np.zeros((n, m + b))
    H = np.zeros((m + b, m))
    state = {"counter": 0, "replacements": 0}
    # the start block's largest column norm seeds the ||A|| scale of the breakdown test
    anorm = float(np.max(np.linalg.norm(start, axis=0)))
    Q, _, _ = orth_block(np.zeros((n, 0)), start, anorm, seed, state)  # orthonormalise start
    V[:, :b] = Q
    k = 0
    restarts = 0
    nspmm = 0
    while True:
        # (1) update the subspace: block Krylov expansion from block k/b to NB
        for j in range(k // b, nblocks):
            W = spmm(V[:, j * b:(j + 1) * b])
            nspmm += 1
            anorm = max(anorm, float(np.max(blockops.mv_norm(W))))
            Q, G, R = orth_block(V[:, :(j + 1) * b], W, anorm, seed, state)
            H[:(j + 1) * b, j * b:(j + 1) * b] = G
            H[(j + 1) * b:(j + 2) * b, j * b:(j + 1) * b] = R
            V[:, (j + 1) * b:(j + 2) * b] = Q
        # (2) projected eigenproblem
        T = 0.5 * (H[:m, :m] + H[:m, :m].T)
        theta, Y = core.jacobi(T)
        order = sort_order(theta, which)
        theta, Y = theta[order], Y[:, order]
        anorm = max(anorm, float(np.max(np.abs(theta))))
        # (3)-(4) residual estimate and convergence test
        rho = np.linalg.norm(H[m:m + b, :m] @ Y, axis=0)
        scale = np.maximum(np.abs(theta), SMALL_THETA * np.max(np.abs(theta)))
        conv = rho <= tol * scale
        nconv = int(np.sum(conv[:nev]))
        if nconv == nev or restarts == max_restarts:
            X = V[:, :m] @ Y[:, :nev]
            AX = np.concatenate([spmm(X[:, c:c + b]) for c in range(0, nev, b)], axis=1)
            nspmm += -(-nev // b)
            resid = blockops.mv_norm(blockops.mv_add_mv(1.0, AX, -1.0,
                                                        blockops.mv_scale2(X, theta[:nev])))
            good = bool(np.all(resid <= tol * scale[:nev]))
            if (nconv == nev and good) or restarts == max_restarts:
                X = X * np.where(X[np.argmax(np.abs(X), axis=0), np.arange(nev)] < 0, -1.0, 1.0)
                return Result(theta[:nev].copy(), X, nconv == nev and good,
                              nconv if good else int(np.sum(resid <= tol * scale[:nev])),
                              restarts, nspmm, rho[:nev].copy(), resid, anorm,
                              state["replacements"])
        # restart: keep the first k Ritz vectors
        k = restart_size(nev, b, m)
        Bt = H[m:m + b, :m] @ Y[:, :k]
        V[:, :k] = V[:, :m] @ Y[:, :k]
        V[:, k:k + b] = V[:, m:m + b]
        V[:, k + b:] = 0.0
        H[:] = 0.0
        H[:k, :k] = np.diag(theta[:k])
        H[k:k + b, :k] = Bt
        restarts += 1
