"""GPU parity of the Table 1 block operations and the re-orthogonalisation step against the
oracle (numpy FP64 on the same inputs).

Bounds: a k-term FP64 sum errs by at most ~k u |terms|; the kernels sum <= 64 rows per lane
and then combine in FP64, so FP64 results are held to 1e-13 and FP32 ones to 1e-5 of the
absolute-value product (|V|^T |W|, |V| |C| + |beta W|).
"""
import numpy as np
import pytest

import graphgen
import paper_1602_01421_gb300 as fe
from oracle import bks, blockops, rng
from tests.gpu_util import to_dev, torch

pytestmark = pytest.mark.gpu
NP = {"f32": np.float32, "f64": np.float64}
TOL = {"f32": 1e-5, "f64": 1e-13}


def _blocks(nv, n, bv, seed, dtype):
    return graphgen.normal_block(nv * n, bv, seed=seed, dtype=dtype).reshape(nv, n, bv)


def _as_tall(V):
    nv, n, bv = V.shape
    return np.concatenate([V[j] for j in range(nv)], axis=1).astype(np.float64)  # n x nv*bv


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n,nv,bv,bw", [(1, 1, 1, 1), (1000, 1, 4, 4), (5003, 9, 4, 4),
                                        (70001, 17, 4, 4), (33000, 5, 8, 8), (20000, 3, 16, 16),
                                        (12345, 2, 2, 8), (4099, 32, 1, 2), (9001, 128, 4, 4)])
def test_gram_parity(prec, n, nv, bv, bw):
    V = _blocks(nv, n, bv, 1, NP[prec])
    W = graphgen.normal_block(n, bw, seed=2, dtype=NP[prec])
    G = fe.block_gram(to_dev(V), to_dev(W), alpha=0.5).cpu().numpy()
    Vt, W64 = _as_tall(V), W.astype(np.float64)
    ref = blockops.mv_trans_mv(0.5, Vt, W64)
    bound = TOL[prec] * 0.5 * (np.abs(Vt).T @ np.abs(W64)) + 1e-300
    assert np.all(np.abs(G - ref) <= bound)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n,nv,bv,bw", [(1, 1, 1, 1), (5003, 9, 4, 4), (70001, 16, 4, 4),
                                        (33000, 8, 8, 8), (2000, 2, 16, 16), (999, 0, 4, 4),
                                        (9001, 128, 4, 4)])
@pytest.mark.parametrize("alpha,beta", [(-1.0, 1.0), (0.25, 0.0), (2.0, -3.0)])
def test_update_parity(prec, n, nv, bv, bw, alpha, beta):
    t = torch()
    V = _blocks(max(nv, 1), n, bv, 3, NP[prec])[:nv] if nv else None
    C = np.random.default_rng(4).standard_normal((max(nv, 1) * bv, bw))[: nv * bv]
    W = graphgen.normal_block(n, bw, seed=5, dtype=NP[prec])
    Wd = to_dev(W)
    fe.block_update(None if V is None else to_dev(V), to_dev(C), Wd, alpha, beta)
    got = Wd.cpu().numpy().astype(np.float64)
    W64 = W.astype(np.float64)
    if nv:
        Vt = _as_tall(V)
        ref = blockops.mv_times_mat_add_mv(alpha, Vt, C, beta, W64)
        mag = np.abs(alpha) * (np.abs(Vt) @ np.abs(C)) + np.abs(beta * W64)
    else:
        ref = blockops.mv_scale1(beta, W64)
        mag = np.abs(beta * W64)
    k = nv * bv + bw + 2
    rel = {"f32": 6e-8, "f64": 1.2e-16}[prec] * k * 2
    assert np.all(np.abs(got - ref) <= rel * mag + 1e-300)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n,nv,b", [(1, 0, 1), (999, 0, 4), (5003, 3, 4), (70001, 7, 4),
                                    (4099, 8, 4), (33000, 12, 2), (20000, 17, 4), (7777, 5, 8),
                                    (3000, 15, 1), (6001, 128, 4)])
@pytest.mark.parametrize("alpha,beta", [(-1.0, 1.0), (0.5, -2.0)])
def test_update_gram_parity(prec, n, nv, b, alpha, beta):
    """fe_block_update_gram = op1 then op3 on the updated block (oracle: the two Table 1
    operations one after the other, FP64).  Shapes span one warp per tile (<= 16 tiles: block
    of 32 x tiles threads), the per-range reduction (17 blocks), ragged row tails."""
    V = _blocks(max(nv, 1), n, b, 6, NP[prec])[:nv] if nv else None
    C = np.random.default_rng(7).standard_normal((max(nv, 1) * b, b))[: nv * b]
    W = graphgen.normal_block(n, b, seed=8, dtype=NP[prec])
    Wd = to_dev(W)
    G = fe.block_update_gram(None if V is None else to_dev(V), to_dev(C), Wd, alpha, beta)
    got_w = Wd.cpu().numpy().astype(np.float64)
    got_g = G.cpu().numpy()
    W64 = W.astype(np.float64)
    if nv:
        Vt = _as_tall(V)
        ref_w = blockops.mv_times_mat_add_mv(alpha, Vt, C, beta, W64)
        mag = np.abs(alpha) * (np.abs(Vt) @ np.abs(C)) + np.abs(beta * W64)
    else:
        Vt = np.zeros((n, 0))
        ref_w = blockops.mv_scale1(beta, W64)
        mag = np.abs(beta * W64)
    k = nv * b + b + 2
    rel = {"f32": 6e-8, "f64": 1.2e-16}[prec] * k * 2
    assert np.all(np.abs(got_w - ref_w) <= rel * mag + 1e-300)
    # Gram of [V; W_new] against W_new, from the kernel's own W_new (the update's rounding is
    # checked above): bound by |[V W]|^T |W| like the Gram test
    VW = np.concatenate([Vt, got_w], axis=1)
    ref_g = blockops.mv_trans_mv(1.0, VW, got_w)
    bound = TOL[prec] * (np.abs(VW).T @ np.abs(got_w)) + 1e-300
    assert got_g.shape == ((nv + 1) * b, b)
    assert np.all(np.abs(got_g - ref_g) <= bound)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_random_normal_matches_oracle_generator(prec):
    t = torch()
    X = fe.random_normal(10007, 4, dtype=t.float32 if prec == "f32" else t.float64, seed=7,
                         stream=4, offset=123).cpu().numpy()
    ref = rng.normal_block(10007, 4, seed=7, stream=4, offset=123)
    assert np.allclose(X, ref, rtol={"f32": 1e-6, "f64": 1e-13}[prec], atol={"f32": 1e-6, "f64": 1e-13}[prec])


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n,nv,b", [(20000, 0, 4), (20000, 3, 4), (50001, 7, 8), (9000, 2, 16),
                                    (3000, 12, 1)])
def test_orth_matches_oracle(prec, n, nv, b):
    """CGS2 + CholQR2 (Section 3.1 re-orthogonalisation) vs oracle.bks.orth_block."""
    r = np.random.default_rng(nv * 100 + b)
    Vt, _ = np.linalg.qr(r.standard_normal((n, max(nv, 1) * b)))
    Vt = Vt[:, : nv * b]
    V = np.stack([Vt[:, j * b:(j + 1) * b] for j in range(nv)]) if nv else None
    W = r.standard_normal((n, b)) + (Vt @ r.standard_normal((nv * b, b)) if nv else 0.0)
    Wd = to_dev(W.astype(NP[prec]))
    G, R, rep = fe.block_orth(None if V is None else to_dev(V.astype(NP[prec])), Wd, anorm=10.0)
    Q = Wd.cpu().numpy().astype(np.float64)
    G, R = G.cpu().numpy(), R.cpu().numpy()
    W64 = W.astype(NP[prec]).astype(np.float64)
    Vq = Vt.astype(NP[prec]).astype(np.float64)
    Qo, Go, Ro = bks.orth_block(Vq if nv else np.zeros((n, 0)), W64, 10.0, 1,
                                {"counter": 0, "replacements": 0})
    tol = {"f32": 2e-5, "f64": 1e-11}[prec]
    assert rep == 0
    assert np.allclose(R, Ro, rtol=tol, atol=tol * np.abs(Ro).max())
    if nv:
        assert np.allclose(G, Go, rtol=tol, atol=tol * np.abs(Go).max())
    assert np.abs(Q.T @ Q - np.eye(b)).max() < {"f32": 1e-5, "f64": 1e-13}[prec]
    if nv:
        assert np.abs(Vq.T @ Q).max() < {"f32": 1e-5, "f64": 1e-13}[prec]
    recon = (Vq @ G if nv else 0.0) + Q @ R
    assert np.abs(recon - W64).max() < {"f32": 1e-4, "f64": 1e-11}[prec] * np.abs(W64).max()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_orth_breakdown_replaces_columns(prec):
    """W with two columns inside span(V) and one duplicate: three random replacements,
    R[i][i] = 0 for them, output still orthonormal and orthogonal to V."""
    n, b, nv = 4000, 4, 2
    r = np.random.default_rng(3)
    Vt, _ = np.linalg.qr(r.standard_normal((n, nv * b)))
    V = np.stack([Vt[:, j * b:(j + 1) * b] for j in range(nv)])
    W = np.empty((n, b))
    W[:, 0] = r.standard_normal(n)
    W[:, 1] = Vt @ r.standard_normal(nv * b)
    W[:, 2] = 2.0 * W[:, 0]
    W[:, 3] = Vt @ r.standard_normal(nv * b)
    Wd = to_dev(W.astype(NP[prec]))
    G, R, rep = fe.block_orth(to_dev(V.astype(NP[prec])), Wd, anorm=100.0, seed=5)
    Q = Wd.cpu().numpy().astype(np.float64)
    R = R.cpu().numpy()
    if prec == "f64":
        assert rep == 3
        assert R[1, 1] == 0.0 and R[2, 2] == 0.0 and R[3, 3] == 0.0
    else:
        # FP32 remainders of dependent columns are rounding noise (~1e-7 |w|), far above the
        # 1e-12 ||A|| breakdown level: they are kept as (random) directions, R[i][i] tiny
        assert abs(R[1, 1]) < 1e-5 * abs(R[0, 0]) and abs(R[3, 3]) < 1e-5 * abs(R[0, 0])
    assert np.abs(Q.T @ Q - np.eye(b)).max() < {"f32": 1e-5, "f64": 1e-12}[prec]
    assert np.abs(Vt.T @ Q).max() < {"f32": 1e-5, "f64": 1e-12}[prec]
    recon = Vt @ G.cpu().numpy() + Q @ R
    assert np.abs(recon - W).max() < {"f32": 1e-4, "f64": 1e-10}[prec] * np.abs(W).max()


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("nv,nout,bv", [(128, 64, 4), (64, 100, 4), (32, 128, 2)])
def test_combine_many_blocks_matches_oracle(prec, nv, nout, bv):
    """The restart product with large subspaces (up to 128 input and output blocks, several
    launches of the coefficient-tiled FMA kernel) against the oracle's op1."""
    n = 3001
    V = _blocks(nv, n, bv, 7, NP[prec])
    Y = np.random.default_rng(8).standard_normal((nv * bv, nout * bv))
    out = fe.block_combine(to_dev(V), to_dev(Y), nout, engine="fma").cpu().numpy()
    got = np.concatenate([out[o] for o in range(nout)], axis=1).astype(np.float64)
    Vt = _as_tall(V)
    ref = Vt @ Y
    rel = {"f32": 6e-8, "f64": 1.2e-16}[prec] * (nv * bv + 2) * 2
    assert np.all(np.abs(got - ref) <= rel * (np.abs(Vt) @ np.abs(Y)) + 1e-300)
