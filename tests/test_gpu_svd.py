"""SVD of directed graphs on the GPU (fe_spmm_t, fe_svds) against the CPU oracle.

The paper's page graph is directed, so its solver computes singular values through A^T A
(Section 4.3.2).  Targets: A^T X within the SpMM tolerances (FP64 1e-13, FP32 1e-6 relative to
A^T |X|); singular values within 1e-8 relative of the oracle's and of dense SVD; right vectors
with eigen-residual ||A^T A v - sigma^2 v|| <= tol * sigma_1^2, left vectors u = A v / sigma.
"""
import numpy as np
import pytest

import graphgen
import paper_1602_01421_gb300 as fe
from oracle import core, svd
from tests.gpu_util import to_dev, torch

pytestmark = pytest.mark.gpu


def _tcsr(g):
    return graphgen.CSR(g.n, *svd.transpose(g.rowptr, g.colidx))


@pytest.mark.parametrize("prec,rel", [("f64", 1e-13), ("f32", 1e-6)])
@pytest.mark.parametrize("b", [1, 2, 4, 8, 16])
def test_spmm_t_matches_oracle(prec, rel, b):
    g = graphgen.rmat(13, seed=2, directed=True)
    t = _tcsr(g)
    X = graphgen.normal_block(g.n, b, seed=b, dtype=np.float64 if prec == "f64" else np.float32)
    with fe.Csr.from_graph(g) as h:
        assert h.info()["has_transpose"] == 1
        Y = fe.spmm_t(h, to_dev(X)).cpu().numpy()
        Yf = fe.spmm(h, to_dev(X)).cpu().numpy()
    X64 = X.astype(np.float64)
    for csr, got in ((t, Y), (g, Yf)):
        ref = core.spmm(csr.rowptr, csr.colidx, X64)
        bound = rel * core.spmm(csr.rowptr, csr.colidx, np.abs(X64))
        assert np.all(np.abs(got.astype(np.float64) - ref) <= bound)
    # A^T 1 = in-degrees exactly
    ones = np.ones((g.n, 1))
    with fe.Csr.from_graph(g) as h:
        indeg = fe.spmm_t(h, to_dev(ones)).cpu().numpy()[:, 0]
    assert np.array_equal(indeg, np.bincount(g.colidx, minlength=g.n).astype(np.float64))


def test_spmm_t_needs_the_transpose():
    g = graphgen.rmat(10, seed=1, directed=True)
    with fe.Csr.from_graph(g, transpose=False) as h:
        assert h.info()["has_transpose"] == 0
        with pytest.raises(fe.FeError):
            fe.spmm_t(h, to_dev(np.ones((g.n, 4))))
        with pytest.raises(fe.FeError):
            fe.svds(h, 4, 2, 8, 1e-8)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_svds_matches_oracle_and_dense(mode):
    """The paper's page-graph setting on a small directed R-MAT: block 2, 2 x nsv blocks."""
    g = graphgen.rmat(12, seed=3, directed=True)
    ref = svd.svds(g.rowptr, g.colidx, 8, 2, 16, 1e-8, seed=1)
    assert ref.eig.converged
    A = g.dense()
    s = np.linalg.svd(A, compute_uv=False)
    with fe.Csr.from_graph(g) as h:
        sv, V, U, st = fe.svds(h, 8, 2, 16, 1e-8, seed=1, mode=mode)
    assert st["converged"]
    assert np.allclose(sv, ref.svals, rtol=1e-8, atol=0)
    assert np.allclose(sv, s[:8], rtol=1e-8, atol=0)
    V, U = V.cpu().numpy(), U.cpu().numpy()
    assert np.abs(V.T @ V - np.eye(8)).max() < 1e-10
    r = np.linalg.norm(A.T @ (A @ V) - V * sv ** 2, axis=0)
    assert np.all(r <= 1e-8 * s[0] ** 2 * 1.001)
    assert np.abs(A @ V - U * sv).max() <= 1e-12 * s[0]
    idx = np.argmax(np.abs(V), axis=0)
    assert np.all(V[idx, np.arange(8)] > 0)
    # the right singular subspace agrees with the oracle's
    c = np.linalg.svd(ref.right.T @ V, compute_uv=False)
    assert c.min() > 1 - 1e-6


@pytest.mark.parametrize("fmt", ["plain", "packed"])
def test_svds_semi_external(fmt):
    """The paper's setting for its directed page graph: the SVD with the matrix (and here its
    transpose) streamed in panels from pinned host memory."""
    g = graphgen.rmat(14, seed=7, directed=True)
    t = _tcsr(g)
    ref = svd.svds(g.rowptr, g.colidx, 6, 2, 12, 1e-8, seed=1)
    X = graphgen.normal_block(g.n, 4, seed=2)
    with fe.Csr.from_graph(g, device_mem_cap_bytes=1 << 18, index_format=fmt) as hs:
        info = hs.info()
        assert info["semi_external"] == 1 and info["has_transpose"] == 1 and info["panels"] > 2
        Yt = fe.spmm_t(hs, to_dev(X)).cpu().numpy()
        sv, V, U, st = fe.svds(hs, 6, 2, 12, 1e-8, seed=1)
    ref_t = core.spmm(t.rowptr, t.colidx, X)
    assert np.all(np.abs(Yt - ref_t) <= 1e-13 * core.spmm(t.rowptr, t.colidx, np.abs(X)))
    assert st["converged"]
    assert np.allclose(sv, ref.svals, rtol=1e-8)
    A = g.dense()
    V, U = V.cpu().numpy(), U.cpu().numpy()
    assert np.abs(A @ V - U * sv).max() <= 1e-12 * sv[0]
    r = np.linalg.norm(A.T @ (A @ V) - V * sv ** 2, axis=0)
    assert np.all(r <= 1e-8 * sv[0] ** 2 * 1.001)


def test_svds_same_start_same_iteration_as_oracle():
    g = graphgen.rmat(11, seed=4, directed=True)
    start = graphgen.normal_block(g.n, 4, seed=5)
    ref = svd.svds(g.rowptr, g.colidx, 6, 4, 6, 1e-9, start=start)
    with fe.Csr.from_graph(g) as h:
        sv, V, U, st = fe.svds(h, 6, 4, 6, 1e-9, start=to_dev(start))
    assert np.allclose(sv, ref.svals, rtol=5e-9)
    assert abs(st["restarts"] - ref.eig.restarts) <= max(2, ref.eig.restarts // 10)


def test_svds_closed_forms():
    n = 60
    g = graphgen.transitive_tournament(n)
    with fe.Csr.from_graph(g) as h:
        sv, V, U, st = fe.svds(h, 6, 2, 10, 1e-11)
    k = np.arange(1, 7)
    assert np.allclose(sv, 1.0 / (2.0 * np.sin((2 * k - 1) * np.pi / (4 * (n - 1) + 2))), rtol=1e-10)
    g = graphgen.complete_bipartite_directed(7, 11)
    with fe.Csr.from_graph(g) as h:
        sv, V, U, st = fe.svds(h, 1, 2, 4, 1e-12)
    assert np.isclose(sv[0], np.sqrt(77.0), rtol=1e-12)
    g = graphgen.directed_cycle(64)
    with fe.Csr.from_graph(g) as h:
        sv, V, U, st = fe.svds(h, 4, 2, 4, 1e-10)
    assert np.allclose(sv, 1.0, atol=1e-12) and st["replacements"] > 0


def test_svds_vectors_optional_and_learned_start_rejected():
    g = graphgen.rmat(11, seed=6, directed=True)
    with fe.Csr.from_graph(g) as h:
        sv, V, U, st = fe.svds(h, 4, 2, 8, 1e-8, return_vectors=False)
        sv2, V2, U2, _ = fe.svds(h, 4, 2, 8, 1e-8)
        assert V is None and U is None and np.allclose(sv, sv2, rtol=1e-12)
        lib = fe.load()
        from paper_1602_01421_gb300 import _lib
        import ctypes
        o = _lib.EigsOpts()
        lib.fe_eigs_opts_default(ctypes.byref(o))
        o.start = _lib.START["learned"]
        w = torch().zeros(1000, dtype=torch().float32, device="cuda")
        o.mlp_weights = w.data_ptr()
        out = np.zeros(4)
        rc = lib.fe_svds(h.handle, 4, 2, 8, 1e-8, ctypes.byref(o),
                         out.ctypes.data_as(ctypes.c_void_p), None, None, None)
        assert rc == _lib.FE_ERR_INVALID


def test_svds_host_memory_subspace_same_results():
    g = graphgen.rmat(12, seed=3, directed=True)
    with fe.Csr.from_graph(g) as h:
        sv_d, V_d, U_d, st_d = fe.svds(h, 8, 2, 16, 1e-8, seed=1)
        sv_h, V_h, U_h, st_h = fe.svds(h, 8, 2, 16, 1e-8, seed=1, subspace="host")
    assert st_h["converged"] and np.array_equal(sv_h, sv_d)
    assert np.array_equal(V_h.cpu().numpy(), V_d.cpu().numpy())
    assert np.array_equal(U_h.cpu().numpy(), U_d.cpu().numpy())
