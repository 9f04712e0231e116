"""GPU Block Krylov-Schur (fe_eigs) against closed-form spectra, brute force and the oracle.

Targets: eigenvalues within 1e-8 relative of the oracle's, residual ||A x - theta x|| <=
tol * ||A|| (checked with the oracle's SpMM on the returned vectors), vectors orthonormal,
eigenvectors compared by subspace angle where eigenvalues cluster.
"""
import numpy as np
import pytest

import graphgen
import paper_1602_01421_gb300 as fe
from oracle import bks, core
from tests import closed_forms
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


def _check_pairs(g, evals, X, tol, anorm):
    X = X.cpu().numpy()
    assert np.abs(X.T @ X - np.eye(X.shape[1])).max() < 1e-10
    r = np.linalg.norm(core.spmm(g.rowptr, g.colidx, X) - X * evals, axis=0)
    assert np.all(r <= tol * anorm * 1.001), r
    # sign convention: largest-magnitude entry positive
    idx = np.argmax(np.abs(X), axis=0)
    assert np.all(X[idx, np.arange(X.shape[1])] > 0)


@pytest.mark.parametrize("case", closed_forms.cases(), ids=lambda c: "-".join(map(str, c)))
def test_eigs_closed_form_spectra(case):
    fam, size, nev, b, nb, which = case
    g = closed_forms.graph(fam, size)
    with fe.Csr.from_graph(g) as h:
        ev, X, st = fe.eigs(h, nev, b, nb, 1e-10, which, seed=3, max_restarts=3000)
    want = closed_forms.wanted(fam, size, nev, which)
    lam = closed_forms.spectrum(fam, size)
    scale = np.abs(lam).max()
    if which == "LM":
        assert np.allclose(np.sort(np.abs(ev)), np.sort(np.abs(want)), atol=1e-9 * scale)
    else:
        assert np.allclose(ev, want, atol=1e-9 * scale)
    assert np.all(np.min(np.abs(ev[:, None] - lam[None, :]), axis=1) < 1e-9 * scale)
    _check_pairs(g, ev, X, 1e-10, scale)


@pytest.mark.parametrize("mode,pass1", [("fp64", "fp32"), ("fp64", "fp64"), ("mixed", "fp32")])
def test_eigs_rmat14_matches_oracle(mode, pass1):
    """The benchmark's small configuration: R-MAT scale 14, nev 8 LM, block 4, 8 blocks,
    tol 1e-8, counter-RNG start (seed 1); the FP64 subspace with the first Gram-Schmidt pass's
    Gram in FP32 or FP64 arithmetic."""
    g = graphgen.rmat(14, seed=1)
    ref = bks.block_krylov_schur(g.rowptr, g.colidx, 8, 4, 8, 1e-8, "LM", seed=1)
    assert ref.converged
    with fe.Csr.from_graph(g) as h:
        ev, X, st = fe.eigs(h, 8, 4, 8, 1e-8, "LM", mode=mode, seed=1, orth_pass1=pass1)
    assert st["converged"] and st["nconv"] == 8
    assert np.allclose(ev, ref.evals, rtol=1e-8, atol=0)
    _check_pairs(g, ev, X, 1e-8, ref.evals[0])
    # subspace of the 8 vectors agrees with the oracle's (principal angles)
    s = np.linalg.svd(ref.evecs.T @ X.cpu().numpy(), compute_uv=False)
    assert s.min() > 1 - 1e-6


@pytest.mark.parametrize("name,which", [("rmat14", "LM"), ("rmat12", "LA")])
def test_eigs_local_first_pass_matches_full(name, which):
    """First Gram-Schmidt pass from the projected matrix's symmetry (orth_local, the default)
    against the full first pass: the same eigenvalues (to 1e-10 relative), both converged,
    residuals within tolerance by the oracle's SpMM, restart counts within a few."""
    g = graphgen.rmat(14 if name == "rmat14" else 12, seed=2)
    with fe.Csr.from_graph(g) as h:
        ev1, X1, st1 = fe.eigs(h, 8, 4, 8, 1e-8, which, seed=3)
        ev0, X0, st0 = fe.eigs(h, 8, 4, 8, 1e-8, which, seed=3, orth_local=False)
    assert st1["converged"] and st0["converged"]
    assert np.allclose(ev1, ev0, rtol=1e-10, atol=1e-10 * np.abs(ev0).max())
    _check_pairs(g, ev1, X1, 1e-8, np.abs(ev0).max())
    assert abs(st1["restarts"] - st0["restarts"]) <= max(5, st0["restarts"] // 5)


def test_eigs_same_start_same_iteration_as_oracle():
    g = graphgen.rmat(12, seed=4)
    start = graphgen.normal_block(g.n, 4, seed=9)
    ref = bks.block_krylov_schur(g.rowptr, g.colidx, 6, 4, 6, 1e-9, "LA", start=start)
    with fe.Csr.from_graph(g) as h:
        ev, X, st = fe.eigs(h, 6, 4, 6, 1e-9, "LA", start=to_dev(start))
    assert np.allclose(ev, ref.evals, rtol=1e-9 * 5)
    assert abs(st["restarts"] - ref.restarts) <= max(2, ref.restarts // 10)
    assert st["spmm_blocks"] > 0


@pytest.mark.parametrize("which", ["LA", "SA", "LM"])
def test_eigs_matches_dense_brute_force(which):
    g = graphgen.rmat(11, seed=2)
    lam = np.linalg.eigvalsh(g.dense())
    want = lam[bks.sort_order(lam, which)][:5]
    with fe.Csr.from_graph(g) as h:
        ev, X, st = fe.eigs(h, 5, 2, 10, 1e-9, which, seed=4, max_restarts=2000)
    scale = np.abs(lam).max()
    assert np.allclose(ev, want, rtol=1e-8, atol=1e-10 * scale)
    _check_pairs(g, ev, X, 1e-9, scale)


def test_eigs_breakdown_complete_graph():
    g = graphgen.complete(60)
    with fe.Csr.from_graph(g) as h:
        ev, X, st = fe.eigs(h, 3, 4, 4, 1e-10, "LM", seed=2)
    assert st["replacements"] > 0
    assert np.allclose(ev, [59.0, -1.0, -1.0], atol=1e-9)


def test_eigs_noconverge_returns_partial():
    g = graphgen.rmat(13, seed=5)
    with fe.Csr.from_graph(g) as h:
        ev, X, st = fe.eigs(h, 8, 4, 4, 1e-12, "LM", max_restarts=1, raise_on_noconverge=False)
    assert not st["converged"] and st["restarts"] == 1 and 0 <= st["nconv"] < 8
    assert np.all(np.isfinite(ev)) and ev[0] > 0
    with fe.Csr.from_graph(g) as h:
        with pytest.raises(fe.FeError) as e:
            fe.eigs(h, 8, 4, 4, 1e-12, "LM", max_restarts=1)
    assert e.value.code == -4


def test_eigs_rejects_bad_sizes():
    g = graphgen.cycle(30)
    with fe.Csr.from_graph(g) as h:
        for args in [(8, 4, 2), (2, 3, 4), (2, 4, 7), (0, 4, 4)]:
            with pytest.raises(fe.FeError):
                fe.eigs(h, *args)


@pytest.mark.slow
def test_eigs_rmat22_full_size():
    """The benchmark solve (R-MAT scale 22, nev 8, block 4, 8 blocks, tol 1e-8): residuals by
    the oracle's SpMM, bounds, and FP64 vs mixed agreement."""
    g = graphgen.rmat(22, seed=1)
    deg = g.degrees()
    with fe.Csr.from_graph(g) as h:
        ev, X, st = fe.eigs(h, 8, 4, 8, 1e-8, "LM", seed=1, max_restarts=5000)
        ev2, X2, st2 = fe.eigs(h, 8, 4, 8, 1e-8, "LM", mode="mixed", seed=1, max_restarts=5000)
    assert st["converged"] and st2["converged"]
    assert deg.mean() <= ev[0] <= deg.max() and ev[0] >= np.sqrt(deg.max())
    _check_pairs(g, ev, X, 1e-8, ev[0])
    _check_pairs(g, ev2, X2, 1e-8, ev2[0])
    assert np.allclose(ev, ev2, rtol=1e-8)


@pytest.mark.parametrize("nev,b,nb,which", [(4, 1, 12, "LM"), (8, 8, 4, "LA"), (16, 16, 3, "LM"),
                                            (3, 2, 9, "SA")])
def test_eigs_block_sizes_match_dense(nev, b, nb, which):
    g = graphgen.rmat(12, seed=7)
    lam = np.linalg.eigvalsh(g.dense())
    want = lam[bks.sort_order(lam, which)][:nev]
    with fe.Csr.from_graph(g) as h:
        ev, X, st = fe.eigs(h, nev, b, nb, 1e-9, which, seed=2, max_restarts=3000)
    scale = np.abs(lam).max()
    assert np.allclose(ev, want, rtol=1e-8, atol=1e-10 * scale)
    _check_pairs(g, ev, X, 1e-9, scale)


def test_mixed_block8_subspace64_matches_oracle():
    """The mixed-precision configuration's shape (block 8, 8 blocks) on a small graph."""
    g = graphgen.rmat(13, seed=3)
    ref = bks.block_krylov_schur(g.rowptr, g.colidx, 8, 8, 8, 1e-8, "LM", seed=1)
    with fe.Csr.from_graph(g) as h:
        ev, X, st = fe.eigs(h, 8, 8, 8, 1e-8, "LM", mode="mixed", seed=1)
    assert st["converged"] and st["spmm_blocks_fp32"] > 0
    assert np.allclose(ev, ref.evals, rtol=1e-8)
    _check_pairs(g, ev, X, 1e-8, ref.evals[0])


def test_mixed_on_semi_external_matrix():
    g = graphgen.rmat(14, seed=1)
    ref = bks.block_krylov_schur(g.rowptr, g.colidx, 8, 4, 8, 1e-8, "LM", seed=1)
    with fe.Csr.from_graph(g, device_mem_cap_bytes=1 << 20) as hs:
        ev, X, st = fe.eigs(hs, 8, 4, 8, 1e-8, "LM", mode="mixed", seed=1)
    assert np.allclose(ev, ref.evals, rtol=1e-8)
    _check_pairs(g, ev, X, 1e-8, ref.evals[0])


def test_output_vectors_orthonormal_every_time():
    """Regression: the sign normalisation must not race with its own flips (n = 32768 gives
    64 reduction blocks per column); every output must be orthonormal with a positive
    largest-magnitude entry, on repeated solves."""
    g = graphgen.rmat(15, seed=2)
    with fe.Csr.from_graph(g) as h:
        for rep in range(4):
            ev, X, st = fe.eigs(h, 8, 4, 8, 1e-8, "LM", seed=1 + rep, max_restarts=0,
                                raise_on_noconverge=False)
            Xh = X.cpu().numpy()
            assert np.abs(Xh.T @ Xh - np.eye(8)).max() < 1e-12
            idx = np.argmax(np.abs(Xh), axis=0)
            assert np.all(Xh[idx, np.arange(8)] > 0)


def test_fp32_first_pass_keeps_the_krylov_relation():
    """With the first pass's Gram in FP32 arithmetic the FP64 solve still reaches residuals of
    tol * ||A|| on a graph whose spectrum has a tight cluster (R-MAT scale 16), in about the
    same number of restarts as the all-FP64 pass, with orthonormal vectors."""
    g = graphgen.rmat(16, seed=2)
    out = {}
    with fe.Csr.from_graph(g) as h:
        for p1 in ("fp32", "fp64"):
            out[p1] = fe.eigs(h, 8, 4, 8, 1e-9, "LM", seed=1, orth_pass1=p1, max_restarts=5000)
    (e32, X32, s32), (e64, X64, s64) = out["fp32"], out["fp64"]
    assert s32["converged"] and s64["converged"]
    assert np.allclose(e32, e64, rtol=1e-9, atol=0)
    _check_pairs(g, e32, X32, 1e-9, abs(e64[0]))
    assert s32["restarts"] <= 1.2 * s64["restarts"] + 5


def test_mixed_tolerance_below_fp32_floor_hands_over():
    """A mixed-mode FP32 tolerance below what FP32 can reach (1e-8 relative) must not keep the
    FP32 phase running to max_restarts: it stops once its residual ratio stops halving, and the
    FP64 phase reaches the same eigenpairs as the plain FP64 solve."""
    g = graphgen.rmat(14, seed=1)
    with fe.Csr.from_graph(g) as h:
        ev0, _, st0 = fe.eigs(h, 8, 4, 8, 1e-8, "LM", seed=1)
        ev1, X1, st1 = fe.eigs(h, 8, 4, 8, 1e-8, "LM", mode="mixed", mixed_tol=1e-8, seed=1,
                               max_restarts=5000)
    assert st1["converged"]
    assert st1["restarts_fp32"] < 5000 and st1["restarts"] < 5000
    assert np.allclose(ev1, ev0, rtol=1e-8)
    _check_pairs(g, ev1, X1, 1e-8, abs(ev0[0]))


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_host_memory_subspace_same_results(mode):
    """The subspace blocks in pinned host memory (read and written by the kernels over the
    CPU-GPU link, the newest block cached on the device) give the same iteration and the same
    results as the device-resident subspace, bit for bit."""
    g = graphgen.rmat(14, seed=1)
    with fe.Csr.from_graph(g) as h:
        ev_d, X_d, st_d = fe.eigs(h, 8, 4, 8, 1e-8, "LM", seed=1, mode=mode)
        ev_h, X_h, st_h = fe.eigs(h, 8, 4, 8, 1e-8, "LM", seed=1, mode=mode, subspace="host")
    assert st_h["converged"] and st_h["restarts"] == st_d["restarts"]
    assert np.array_equal(ev_h, ev_d)
    assert np.array_equal(X_h.cpu().numpy(), X_d.cpu().numpy())


def test_fully_external_solve_matches_oracle():
    """The paper's semi-external eigensolver in full: the CSR streamed in panels from pinned host
    memory and the subspace in host memory, only the newest block and the small matrices on
    the device; checked against the oracle."""
    g = graphgen.rmat(14, seed=1)
    ref = bks.block_krylov_schur(g.rowptr, g.colidx, 8, 4, 8, 1e-8, "LM", seed=1)
    with fe.Csr.from_graph(g, device_mem_cap_bytes=1 << 20) as hs:
        assert hs.info()["semi_external"] == 1
        ev, X, st = fe.eigs(hs, 8, 4, 8, 1e-8, "LM", seed=1, subspace="host")
    assert st["converged"]
    assert np.allclose(ev, ref.evals, rtol=1e-8)
    _check_pairs(g, ev, X, 1e-8, ref.evals[0])
