"""Pins for the CPU oracle: each test checks it against something other than itself
(closed forms, brute force, constructions with known answers, published reference outputs)."""
import math
import os

import numpy as np
import pytest

import graphgen
from oracle import blockops, bks, core, rng
from tests import closed_forms

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ---------------------------------------------------------------- SpMM (Section 3.3)
@pytest.mark.parametrize("maker", [lambda: graphgen.rmat(10, seed=3),
                                   lambda: graphgen.erdos_renyi(1500, 7.0, seed=2),
                                   lambda: graphgen.star(300),
                                   lambda: graphgen.disjoint_union(graphgen.cycle(50),
                                                                   graphgen.complete(30))])
@pytest.mark.parametrize("b", [1, 2, 4, 8, 16])
def test_spmm_matches_dense_brute_force(maker, b):
    g = maker()
    X = graphgen.normal_block(g.n, b, seed=b)
    Y = core.spmm(g.rowptr, g.colidx, X)
    Yd = g.dense() @ X
    bound = 1e-14 * (g.dense() @ np.abs(X)) + 1e-300
    assert np.all(np.abs(Y - Yd) <= bound)


def test_spmm_ones_is_degree_exactly():
    g = graphgen.rmat(12, seed=5)
    Y = core.spmm(g.rowptr, g.colidx, np.ones((g.n, 3)))
    assert np.array_equal(Y, np.repeat(g.degrees()[:, None].astype(np.float64), 3, axis=1))


def test_spmm_float32_input_is_widened_exactly():
    g = graphgen.rmat(10, seed=7)
    X32 = graphgen.normal_block(g.n, 4, seed=1, dtype=np.float32)
    Y = core.spmm(g.rowptr, g.colidx, X32)
    Yd = g.dense() @ X32.astype(np.float64)
    assert np.allclose(Y, Yd, rtol=0, atol=1e-12)


def test_spmm_rows_and_empty_rows():
    g = graphgen.disjoint_union(graphgen.star(20), graphgen.from_edges(5, [], [], "empty5"))
    X = graphgen.normal_block(g.n, 2, seed=9)
    Y = core.spmm(g.rowptr, g.colidx, X)
    assert np.all(Y[20:] == 0.0)                      # isolated vertices: zero rows
    assert np.allclose(Y[0], X[1:20].sum(axis=0))     # hub row = sum of its leaves
    rows = np.array([3, 0, 24, 0])
    assert np.array_equal(core.spmm_rows(g.rowptr, g.colidx, X, rows), Y[rows])


def test_spmm_is_linear_and_symmetric():
    """For symmetric A: <A x, y> = <x, A y> and A(ax + y) = a Ax + Ay (brute-force-free)."""
    g = graphgen.rmat(11, seed=11)
    x = graphgen.normal_block(g.n, 1, seed=1)
    y = graphgen.normal_block(g.n, 1, seed=2)
    Ax = core.spmm(g.rowptr, g.colidx, x)
    Ay = core.spmm(g.rowptr, g.colidx, y)
    assert abs(float(Ax[:, 0] @ y[:, 0] - x[:, 0] @ Ay[:, 0])) < 1e-9
    A2 = core.spmm(g.rowptr, g.colidx, 3.0 * x + y)
    assert np.allclose(A2, 3.0 * Ax + Ay, atol=1e-11)


# ---------------------------------------------------------------- Jacobi (Algorithm 1 step 2)
def test_jacobi_2x2_closed_form():
    a, b_, c = 2.0, 1.5, -1.0
    ev, Y = core.jacobi(np.array([[a, b_], [b_, c]]))
    mid, rad = (a + c) / 2, math.hypot((a - c) / 2, b_)
    assert np.allclose(np.sort(ev), [mid - rad, mid + rad], atol=1e-15)


@pytest.mark.parametrize("m", [1, 3, 8, 32, 64])
def test_jacobi_recovers_constructed_spectrum(m):
    r = np.random.default_rng(m)
    Q, _ = np.linalg.qr(r.standard_normal((m, m)))
    lam = np.sort(r.uniform(-5, 5, m))
    lam[: m // 4] = lam[0]            # include a repeated eigenvalue
    T = (Q * lam) @ Q.T
    T = 0.5 * (T + T.T)
    ev, Y = core.jacobi(T)
    assert np.allclose(np.sort(ev), lam, atol=1e-12 * 5 * m)
    assert np.allclose(Y.T @ Y, np.eye(m), atol=1e-13 * m)
    assert np.allclose(T @ Y, Y * ev, atol=1e-12 * m)


def test_jacobi_diagonal_input_is_fixed_point():
    d = np.array([3.0, -1.0, 2.0, 0.0])
    ev, Y = core.jacobi(np.diag(d))
    assert np.array_equal(ev, d) and np.array_equal(Y, np.eye(4))


# ---------------------------------------------------------------- Table 1 block ops
def test_table1_ops_against_definitions_elementwise():
    r = np.random.default_rng(0)
    AA, BB, CC = r.standard_normal((3, 50, 4))
    B = r.standard_normal((4, 4))
    # explicit loops over the index definitions
    op1 = np.array([[2.0 * sum(AA[i, p] * B[p, j] for p in range(4)) - 0.5 * CC[i, j]
                     for j in range(4)] for i in range(50)])
    assert np.allclose(blockops.mv_times_mat_add_mv(2.0, AA, B, -0.5, CC), op1)
    op3 = np.array([[sum(AA[i, p] * BB[i, q] for i in range(50)) for q in range(4)]
                    for p in range(4)])
    assert np.allclose(blockops.mv_trans_mv(1.0, AA, BB), op3)
    assert np.allclose(blockops.mv_dot(AA, BB), [sum(AA[:, j] * BB[:, j]) for j in range(4)])
    assert np.allclose(blockops.mv_norm(AA), [math.sqrt(sum(AA[:, j] ** 2)) for j in range(4)])


def test_cholqr2_orthonormal_and_reconstructs():
    r = np.random.default_rng(1)
    W = r.standard_normal((2000, 8)) @ np.diag(10.0 ** -np.arange(8))   # cond ~1e7
    Q, R, ok = blockops.cholqr2(W, bks.REL_PIVOT, 0.0)
    assert ok
    assert np.abs(Q.T @ Q - np.eye(8)).max() < 1e-13
    assert np.allclose(Q @ R, W, atol=1e-13)
    assert np.allclose(R, np.triu(R))


def test_chol_rejects_dependent_columns():
    r = np.random.default_rng(2)
    W = r.standard_normal((100, 3))
    W = np.concatenate([W, W[:, :1] + 1e-9 * W[:, 1:2]], axis=1)
    _, _, ok = blockops.cholqr(W, bks.REL_PIVOT, 0.0)
    assert not ok


# ---------------------------------------------------------------- counter RNG
def test_splitmix64_reference_outputs():
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        ref = [int(l, 16) for l in f if l.strip() and not l.startswith("#")]
    g = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        got = [int(rng._mix(np.array([g * np.uint64(k)], dtype=np.uint64))[0]) for k in (1, 2, 3, 4)]
    assert got == ref


def test_normal_block_moments_and_determinism():
    z = rng.normal_block(200000, 2, seed=7, stream=4)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1) < 0.01
    assert abs(np.mean(z ** 4) - 3.0) < 0.05          # N(0,1) kurtosis
    assert np.array_equal(z[:10], rng.normal_block(10, 2, seed=7, stream=4))
    assert np.array_equal(rng.normal_block(5, 2, 7, 4, offset=20), z[10:15])


# ---------------------------------------------------------------- Block Krylov-Schur
def _check_eigpairs(g, res, tol, anorm):
    X = res.evecs
    # each restart's V_m Y_k product adds O(m u) to the loss of orthogonality
    assert np.abs(X.T @ X - np.eye(X.shape[1])).max() < max(1e-12, 4e-15 * res.restarts)
    AX = core.spmm(g.rowptr, g.colidx, X)
    r = np.linalg.norm(AX - X * res.evals, axis=0)
    assert np.all(r <= tol * anorm * 1.0001)


@pytest.mark.parametrize("case", closed_forms.cases(), ids=lambda c: "-".join(map(str, c)))
def test_bks_closed_form_spectra(case):
    fam, size, nev, b, nb, which = case
    g = closed_forms.graph(fam, size)
    res = bks.block_krylov_schur(g.rowptr, g.colidx, nev, b, nb, 1e-10, which, seed=3,
                                 max_restarts=2000)
    assert res.converged
    want = closed_forms.wanted(fam, size, nev, which)
    lam = closed_forms.spectrum(fam, size)
    scale = np.abs(lam).max()
    if which == "LM":
        assert np.allclose(np.sort(np.abs(res.evals)), np.sort(np.abs(want)), atol=1e-9 * scale)
    else:
        assert np.allclose(res.evals, want, atol=1e-9 * scale)
    # every Ritz value is an eigenvalue of the closed form
    assert np.all(np.min(np.abs(res.evals[:, None] - lam[None, :]), axis=1) < 1e-9 * scale)
    _check_eigpairs(g, res, 1e-10, scale)


@pytest.mark.parametrize("maker,nev,b,nb,which", [
    (lambda: graphgen.rmat(10, seed=1), 8, 4, 8, "LM"),
    (lambda: graphgen.rmat(11, seed=2), 6, 2, 10, "LA"),
    (lambda: graphgen.erdos_renyi(1800, 10.0, seed=4), 5, 3, 6, "SA"),
    (lambda: graphgen.rmat(10, seed=6, permute=False), 8, 8, 4, "LM"),
])
def test_bks_matches_dense_brute_force(maker, nev, b, nb, which):
    g = maker()
    lam = np.linalg.eigvalsh(g.dense())
    res = bks.block_krylov_schur(g.rowptr, g.colidx, nev, b, nb, 1e-8, which, seed=5)
    assert res.converged
    want = lam[bks.sort_order(lam, which)][:nev]
    scale = np.abs(lam).max()
    assert np.allclose(res.evals, want, rtol=1e-8, atol=1e-10 * scale)
    _check_eigpairs(g, res, 1e-8, scale)


def test_bks_bounds_and_perron_vector():
    g = graphgen.rmat(14, seed=1)
    deg = g.degrees()
    res = bks.block_krylov_schur(g.rowptr, g.colidx, 8, 4, 8, 1e-8, "LM", seed=1)
    assert res.converged
    lam1 = res.evals[0]
    # the Perron root of a nonnegative symmetric matrix: avg degree <= lambda_1 <= max degree,
    # lambda_1 >= sqrt(max degree) (the star around the hub)
    assert deg.mean() <= lam1 <= deg.max()
    assert lam1 >= math.sqrt(deg.max())
    assert np.all(np.abs(res.evals) <= lam1 * (1 + 1e-12))
    # Perron vector: one sign on the giant component (entries outside it are ~0)
    x = res.evecs[:, 0]
    assert x[np.argmax(np.abs(x))] > 0
    assert np.all(x >= -1e-8 * np.abs(x).max())
    _check_eigpairs(g, res, 1e-8, lam1)


def test_bks_breakdown_on_invariant_subspace_uses_replacement():
    # K_n: A V_0 spans at most one new direction, so the block CholQR breaks down at once
    g = graphgen.complete(60)
    res = bks.block_krylov_schur(g.rowptr, g.colidx, 3, 4, 4, 1e-10, "LM", seed=2)
    assert res.converged and res.replacements > 0
    assert np.allclose(res.evals, [59.0, -1.0, -1.0], atol=1e-9)


def test_bks_start_block_and_restart_size():
    assert bks.restart_size(8, 4, 32) == 20
    assert bks.restart_size(8, 8, 64) == 32
    assert bks.restart_size(7, 4, 12) == 8
    g = graphgen.rmat(9, seed=2)
    st = graphgen.normal_block(g.n, 4, seed=11)
    r1 = bks.block_krylov_schur(g.rowptr, g.colidx, 4, 4, 6, 1e-9, "LM", start=st)
    r2 = bks.block_krylov_schur(g.rowptr, g.colidx, 4, 4, 6, 1e-9, "LM", start=st)
    assert np.array_equal(r1.evals, r2.evals) and r1.restarts == r2.restarts


def test_bks_rejects_bad_sizes():
    g = graphgen.cycle(20)
    with pytest.raises(ValueError):
        bks.block_krylov_schur(g.rowptr, g.colidx, 8, 4, 2, 1e-8)
    with pytest.raises(ValueError):
        bks.block_krylov_schur(g.rowptr, g.colidx, 2, 4, 5, 1e-8)   # m + b > n
