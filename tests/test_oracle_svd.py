"""Pins of the oracle's SVD path (oracle/svd.py) against dense linear algebra and closed forms.

Each pin would fail on a plausible slip: a transposed operator (A A instead of A^T A changes
the spectrum), swapped left/right vectors (A v = sigma u fails), a dropped square root, a
wrong transpose (dense comparison), or a sign error in u.
"""
import numpy as np
import pytest

import graphgen
from oracle import svd


def test_transpose_is_the_dense_transpose():
    for g in (graphgen.rmat(9, seed=2, directed=True), graphgen.out_star(17),
              graphgen.transitive_tournament(12), graphgen.complete_bipartite_directed(3, 5)):
        trp, tci = svd.transpose(g.rowptr, g.colidx)
        assert np.array_equal(graphgen.CSR(g.n, trp, tci).dense(), g.dense().T)
        assert np.all(np.diff(trp) >= 0) and trp[-1] == g.nnz
        for i in range(g.n):   # column indices sorted in every row
            assert np.all(np.diff(tci[trp[i]:trp[i + 1]]) > 0)
        r2, c2 = svd.transpose(trp, tci)
        assert np.array_equal(r2, g.rowptr) and np.array_equal(c2, g.colidx)


def test_directed_rmat_is_not_symmetric_and_symmetrises_to_the_undirected_one():
    d = graphgen.rmat(9, seed=4, directed=True).dense()
    u = graphgen.rmat(9, seed=4).dense()
    assert np.abs(d - d.T).sum() > 0 and np.trace(d) == 0
    assert np.array_equal(np.maximum(d, d.T), u)


@pytest.mark.parametrize("scale,seed,nsv,b,nb", [(9, 1, 8, 2, 16), (10, 3, 6, 4, 6), (10, 5, 3, 1, 12)])
def test_svds_matches_dense_svd(scale, seed, nsv, b, nb):
    g = graphgen.rmat(scale, seed=seed, directed=True)
    A = g.dense()
    r = svd.svds(g.rowptr, g.colidx, nsv, b, nb, 1e-10, seed=2, max_restarts=2000)
    assert r.eig.converged
    s = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(r.svals, s[:nsv], rtol=1e-9, atol=0)
    # A v = sigma u exactly by construction, A^T u = sigma v to the eigen-residual
    assert np.abs(A @ r.right - r.left * r.svals).max() <= 1e-12 * s[0]
    resid = np.linalg.norm(A.T @ (A @ r.right) - r.right * r.svals ** 2, axis=0)
    assert np.all(resid <= 1e-10 * s[0] ** 2 * 1.001)
    assert np.abs(r.right.T @ r.right - np.eye(nsv)).max() < 1e-12
    assert np.abs(r.left.T @ r.left - np.eye(nsv)).max() < 1e-8
    idx = np.argmax(np.abs(r.right), axis=0)
    assert np.all(r.right[idx, np.arange(nsv)] > 0)


def test_svds_transitive_tournament_closed_form():
    """i -> j for i < j: the strictly upper triangular all-ones n x n matrix has the singular
    values of the (n-1) x (n-1) triangular all-ones matrix, 1 / (2 sin((2k-1) pi / (4(n-1)+2))),
    plus one zero (its inverse is the bidiagonal difference matrix, whose Gram matrix is the
    tridiagonal [-1 2 -1] with a last diagonal entry of 1)."""
    n = 60
    g = graphgen.transitive_tournament(n)
    r = svd.svds(g.rowptr, g.colidx, 6, 2, 10, 1e-11)
    k = np.arange(1, 7)
    want = 1.0 / (2.0 * np.sin((2 * k - 1) * np.pi / (4 * (n - 1) + 2)))
    assert np.allclose(r.svals, want, rtol=1e-10)


def test_svds_rank_one_closed_forms():
    """Out-star S_n: one non-zero row of n-1 ones, sigma_1 = sqrt(n-1), v = leaves / sqrt(n-1),
    u = e_0.  Directed complete bipartite p -> q: the all-ones p x q block, sigma_1 = sqrt(p q)."""
    g = graphgen.out_star(50)
    r = svd.svds(g.rowptr, g.colidx, 1, 2, 4, 1e-12)
    assert np.isclose(r.svals[0], np.sqrt(49.0), rtol=1e-12)
    want_v = np.r_[0.0, np.ones(49) / 7.0]
    assert np.allclose(r.right[:, 0], want_v, atol=1e-12)
    assert np.allclose(r.left[:, 0], np.eye(50)[0], atol=1e-12)
    g = graphgen.complete_bipartite_directed(7, 11)
    r = svd.svds(g.rowptr, g.colidx, 2, 2, 4, 1e-12)
    assert np.isclose(r.svals[0], np.sqrt(77.0), rtol=1e-12)
    assert abs(r.svals[1]) < 1e-6


def test_svds_permutation_matrix_all_ones():
    """Directed cycle: A is a permutation matrix, A^T A = I, every singular value is 1 (the
    Krylov space is invariant from the start, so the breakdown path supplies the basis)."""
    g = graphgen.directed_cycle(64)
    r = svd.svds(g.rowptr, g.colidx, 4, 2, 4, 1e-10)
    assert np.allclose(r.svals, 1.0, atol=1e-12)
    assert r.eig.replacements > 0
    A = g.dense()
    assert np.abs(A @ r.right - r.left).max() < 1e-12
