"""Many eigenvalues: subspaces beyond the shared-memory Rayleigh-Ritz (96 < m <= 512).

The paper computes larger sets of eigenvalues with block size 4 and as many blocks as
eigenvalues (Section 4.3, the eigensolver settings), so nev = 32 runs with m = 128 and nev = 64
with m = 256; its dense-operation study goes to m = 512 (Section 4.2.2).  Up to m = 160 the
projected problem's eigenvector matrix lives in a device workspace of the one-CTA kernel; above,
FP32 sweeps, FP64 matrix products and cooperative FP64 sweeps take it.  Checked against the
oracle (same iteration), dense brute force, residuals and orthonormality.
"""
import numpy as np
import pytest

import graphgen
import paper_1602_01421_gb300 as fe
from oracle import bks, core
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


def _check_pairs(g, evals, X, tol, anorm):
    X = X.cpu().numpy()
    assert np.abs(X.T @ X - np.eye(X.shape[1])).max() < 1e-10
    AX = np.concatenate([core.spmm(g.rowptr, g.colidx, X[:, c:c + 64]) for c in range(0, X.shape[1], 64)],
                        axis=1)
    r = np.linalg.norm(AX - X * evals, axis=0)
    assert np.all(r <= tol * anorm * 1.001), r
    idx = np.argmax(np.abs(X), axis=0)
    assert np.all(X[idx, np.arange(X.shape[1])] > 0)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_nev32_block4_subspace128_matches_oracle_and_dense(mode):
    """The paper's many-eigenvalue setting: nev 32, block 4, 32 blocks (m = 128)."""
    g = graphgen.rmat(12, seed=5)
    ref = bks.block_krylov_schur(g.rowptr, g.colidx, 32, 4, 32, 1e-8, "LM", seed=1)
    assert ref.converged
    lam = np.linalg.eigvalsh(g.dense())
    want = lam[bks.sort_order(lam, "LM")][:32]
    with fe.Csr.from_graph(g) as h:
        ev, X, st = fe.eigs(h, 32, 4, 32, 1e-8, "LM", seed=1, mode=mode)
    assert st["converged"] and st["nconv"] == 32
    scale = np.abs(lam).max()
    assert np.allclose(ev, ref.evals, rtol=1e-8, atol=1e-10 * scale)
    assert np.allclose(ev, want, rtol=1e-8, atol=1e-10 * scale)
    _check_pairs(g, ev, X, 1e-8, scale)


def test_subspace128_same_start_same_iteration_as_oracle():
    g = graphgen.rmat(12, seed=6)
    start = graphgen.normal_block(g.n, 4, seed=11)
    ref = bks.block_krylov_schur(g.rowptr, g.colidx, 24, 4, 32, 1e-9, "LA", start=start)
    with fe.Csr.from_graph(g) as h:
        ev, X, st = fe.eigs(h, 24, 4, 32, 1e-9, "LA", start=to_dev(start))
    assert np.allclose(ev, ref.evals, rtol=5e-9)
    assert abs(st["restarts"] - ref.restarts) <= max(2, ref.restarts // 10)
    assert abs(st["spmm_blocks"] - ref.spmm_blocks) <= max(8, ref.spmm_blocks // 10)


@pytest.mark.parametrize("nev,b,nb,which", [(16, 8, 20, "LA"), (40, 16, 10, "SA"),
                                            (20, 2, 49, "LM"), (24, 2, 131, "LM")])
def test_largest_subspaces_match_dense(nev, b, nb, which):
    """m = 160 with blocks of 8 and 16 (the one-CTA kernel's largest), block 2 with 49 blocks
    (m = 98); 131 blocks are rejected (more blocks than a block set holds)."""
    g = graphgen.rmat(12, seed=8)
    with fe.Csr.from_graph(g) as h:
        if b * nb > 512 or nb > 130:
            with pytest.raises(fe.FeError):
                fe.eigs(h, nev, b, nb, 1e-9, which)
            return
        ev, X, st = fe.eigs(h, nev, b, nb, 1e-9, which, seed=3, max_restarts=3000)
    lam = np.linalg.eigvalsh(g.dense())
    want = lam[bks.sort_order(lam, which)][:nev]
    scale = np.abs(lam).max()
    assert st["converged"]
    assert np.allclose(ev, want, rtol=1e-8, atol=1e-10 * scale)
    _check_pairs(g, ev, X, 1e-9, scale)


def test_subspace_above_limit_rejected():
    g = graphgen.rmat(11, seed=1)
    with fe.Csr.from_graph(g) as h:
        with pytest.raises(fe.FeError):
            fe.eigs(h, 8, 16, 33, 1e-8, "LM")     # m = 528 > 512


@pytest.mark.parametrize("nev,b,nb,mode", [(64, 4, 64, "fp64"), (64, 4, 64, "mixed"),
                                           (32, 4, 128, "fp64"), (100, 8, 64, "fp64")])
def test_large_subspaces_match_oracle_and_dense(nev, b, nb, mode):
    """m = 256 (nev 64 with the paper's block 4 and as many blocks as eigenvalues) and m = 512
    (block 4 x 128 blocks, block 8 x 64): the cooperative Rayleigh-Ritz and block operations with
    up to 129 blocks, against the oracle's iteration and dense eigvalsh."""
    g = graphgen.rmat(12, seed=5)
    lam = np.linalg.eigvalsh(g.dense())
    want = lam[bks.sort_order(lam, "LM")][:nev]
    scale = np.abs(lam).max()
    with fe.Csr.from_graph(g) as h:
        ev, X, st = fe.eigs(h, nev, b, nb, 1e-8, "LM", seed=1, mode=mode, max_restarts=200)
    assert st["converged"] and st["nconv"] == nev
    assert np.allclose(ev, want, rtol=1e-8, atol=1e-10 * scale)
    _check_pairs(g, ev, X, 1e-8, scale)
    if mode == "fp64" and b * nb == 256:
        ref = bks.block_krylov_schur(g.rowptr, g.colidx, nev, b, nb, 1e-8, "LM", seed=1)
        assert ref.converged
        assert np.allclose(ev, ref.evals, rtol=1e-8, atol=1e-10 * scale)


def test_subspace512_same_start_same_iteration_as_oracle():
    """m = 512 from the same start block: the same Ritz values and about the same number of
    restarts and block SpMMs as the oracle's Block Krylov-Schur."""
    g = graphgen.rmat(11, seed=6)
    start = graphgen.normal_block(g.n, 4, seed=12)
    ref = bks.block_krylov_schur(g.rowptr, g.colidx, 48, 4, 128, 1e-9, "LA", start=start)
    with fe.Csr.from_graph(g) as h:
        ev, X, st = fe.eigs(h, 48, 4, 128, 1e-9, "LA", start=to_dev(start))
    assert ref.converged and st["converged"]
    assert np.allclose(ev, ref.evals, rtol=5e-9)
    assert abs(st["restarts"] - ref.restarts) <= max(2, ref.restarts // 10)
    assert abs(st["spmm_blocks"] - ref.spmm_blocks) <= max(8, ref.spmm_blocks // 10)
