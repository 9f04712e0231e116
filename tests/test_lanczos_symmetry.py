"""CPU pin of the identity behind the solver's first Gram-Schmidt pass from symmetry: with a
symmetric A and the block Krylov-Schur basis of Algorithm 1 (Section 3.1), the coefficient of
an older block v_i in W = A v_j is v_i^T A v_j = (A v_i)^T v_j = H[j][i] -- R_{j-1}^T for
v_{j-1} (the Lanczos recurrence), the restart's coupling B^T for the kept vectors right after
a restart, and zero (to rounding) for every other older block.  The full Gram of the oracle's
own CGS2 (oracle.bks.orth_block) is compared with those entries of H, step by step, through an
expansion, a Krylov-Schur restart and the expansion after it.
"""
import numpy as np

import graphgen
from oracle import bks, core, rng


def _expand(A_mul, V, H, b, j0, nb, anorm, state):
    """Steps j0..nb-1 of the expansion; returns, per step, the full first-pass Gram of W against
    the older blocks and the entries of H that the identity predicts for it."""
    checks = []
    for j in range(j0, nb):
        W = A_mul(V[:, j * b:(j + 1) * b])
        older = V[:, :j * b]
        full = older.T @ W                                # first-pass Gram against v_0..v_{j-1}
        predicted = H[j * b:(j + 1) * b, :j * b].T.copy()  # H[j][i]^T for i < j
        checks.append((j, full, predicted))
        Q, G, R = bks.orth_block(V[:, :(j + 1) * b], W, anorm, 1, state)
        H[:(j + 1) * b, j * b:(j + 1) * b] = G
        H[(j + 1) * b:(j + 2) * b, j * b:(j + 1) * b] = R
        V[:, (j + 1) * b:(j + 2) * b] = Q
    return checks


def test_first_pass_coefficients_are_in_the_projected_matrix():
    g = graphgen.rmat(11, seed=5)
    n, b, nb, nev = g.n, 4, 6, 4
    m = b * nb

    def A_mul(X):
        return core.spmm(g.rowptr, g.colidx, X)

    anorm = float(np.max(np.diff(g.rowptr)))              # >= ||A|| for a 0/1 matrix
    state = {"counter": 0, "replacements": 0}
    V = np.zeros((n, m + b))
    H = np.zeros((m + b, m))
    Q, _, _ = bks.orth_block(np.zeros((n, 0)), rng.normal_block(n, b, 3, 1), anorm, 1, state)
    V[:, :b] = Q
    checks = _expand(A_mul, V, H, b, 0, nb, anorm, state)
    # restart as Algorithm 1 does: keep k Ritz vectors, H <- [diag(theta); B^T]
    T = 0.5 * (H[:m, :m] + H[:m, :m].T)
    theta, Y = core.jacobi(T)
    order = bks.sort_order(theta, "LM")
    theta, Y = theta[order], Y[:, order]
    k = bks.restart_size(nev, b, m)
    Bt = H[m:m + b, :m] @ Y[:, :k]
    V[:, :k] = V[:, :m] @ Y[:, :k]
    V[:, k:k + b] = V[:, m:m + b]
    V[:, k + b:] = 0.0
    H[:] = 0.0
    H[:k, :k] = np.diag(theta[:k])
    H[k:k + b, :k] = Bt
    after = _expand(A_mul, V, H, b, k // b, nb, anorm, state)
    assert state["replacements"] == 0
    scale = anorm
    for j, full, predicted in checks + after:
        if j == 0:
            continue                                       # no older block yet
        # the identity holds to the basis' loss of orthogonality (rounding level here)
        assert np.abs(full - predicted).max() <= 1e-11 * scale, (j, np.abs(full - predicted).max())
    # structure: before the restart only v_{j-1} couples (a plain mistake -- a transposed block,
    # a shifted block row -- breaks these)
    for j, full, predicted in checks:
        if j >= 2:
            assert np.abs(full[:(j - 1) * b]).max() <= 1e-11 * scale
        if j >= 1:
            assert np.abs(full[(j - 1) * b:]).max() > 1e-3          # R_{j-1}^T is not zero
    # right after the restart every kept vector couples through B^T
    j0, full0, _ = after[0]
    assert j0 == k // b
    assert np.allclose(full0, Bt.T, rtol=0, atol=1e-11 * scale)
