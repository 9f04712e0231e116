"""GPU parity of the tensor-core split-product block operations -- fe_block_combine (Table 1
"op1" with several output blocks, the restart product V Y of Section 3.1) against the oracle's
MvTimesMatAddMv, fe_block_gram_ex (Table 1 "op3", MvTransMv) against the oracle's MvTransMv --
and of the solver with tensor-core restart products and second Gram-Schmidt pass against the
oracle's Block Krylov-Schur.

Bounds: the stated worst case |err| <= 2^-49 (K + 1) max_c|V[r][c]| max_c|Y[c][q]| + 2^-52 |ref|
(+ 2^-1022: results below the normal range flush to zero),
and the FP64 block-operation tolerance 1e-13 (|V| |Y|) on N(0,1) data; integer data whose
products fit in 53 bits are reproduced exactly.
"""
import numpy as np
import pytest

import graphgen
import paper_1602_01421_gb300 as fe
from oracle import bks, blockops
from tests.gpu_util import to_dev, torch

pytestmark = pytest.mark.gpu


def _flat(Vb):
    """(nv, n, bv) blocks -> the n x (nv*bv) matrix whose column j*bv + p is block j's column p."""
    nv, n, bv = Vb.shape
    return Vb.transpose(1, 0, 2).reshape(n, nv * bv)


def _run(Vh, Yh, nout, engine="tc"):
    V = to_dev(Vh)
    Y = to_dev(Yh)
    out = fe.block_combine(V, Y, nout, engine=engine)
    torch().cuda.synchronize()
    return _flat(out.cpu().numpy())


def _check(Vh, Yh, got):
    AA = _flat(Vh)
    ref = blockops.mv_times_mat_add_mv(1.0, AA, Yh, 0.0, np.zeros((AA.shape[0], Yh.shape[1])))
    K = AA.shape[1]
    err = np.abs(got - ref)
    # (results below the normal range, 2^-1022, flush to zero)
    stated = (2.0 ** -49 * (K + 1) * np.abs(AA).max(axis=1)[:, None] * np.abs(Yh).max(axis=0)[None, :]
              + 2.0 ** -52 * np.abs(ref) + 2.0 ** -1022)
    assert (err <= stated).all(), f"stated bound: worst {np.max(err - stated):.3e}"
    return err, np.abs(AA) @ np.abs(Yh)


SHAPES = [  # (n, nv, bv, nout)
    (1, 8, 4, 5), (127, 8, 4, 5), (128, 8, 4, 5), (129, 8, 4, 2), (1000, 8, 4, 5),
    (65537, 8, 4, 5), (4099, 16, 4, 8), (3001, 1, 1, 1), (2048, 3, 2, 7), (777, 32, 1, 32),
    (5000, 8, 8, 4), (300, 4, 16, 2), (257, 2, 16, 1), (40000, 9, 4, 3), (1025, 5, 1, 13)]


@pytest.mark.parametrize("shape", SHAPES)
def test_tc_combine_matches_oracle(shape):
    """N(0,1) blocks: per entry within 1e-13 (|V||Y|) and within the stated bound; K up to 64
    (two 32-wide accumulator sets), N up to 32, ragged last 128-row tiles."""
    n, nv, bv, nout = shape
    rng = np.random.default_rng(n + 7 * nv + bv)
    Vh = rng.standard_normal((nv, n, bv))
    Yh = rng.standard_normal((nv * bv, nout * bv))
    got = _run(Vh, Yh, nout)
    err, absprod = _check(Vh, Yh, got)
    assert (err <= 1e-13 * absprod).all()


def test_tc_combine_integers_exact():
    """Integer entries (|x| <= 1000): every product sum fits in 53 bits, and the split products
    are exact, so the result equals the integer product bit for bit."""
    rng = np.random.default_rng(5)
    n, nv, bv, nout = 10007, 8, 4, 5
    Vi = rng.integers(-1000, 1001, (nv, n, bv))
    Yi = rng.integers(-1000, 1001, (nv * bv, nout * bv))
    got = _run(Vi.astype(np.float64), Yi.astype(np.float64), nout)
    exact = _flat(Vi) @ Yi
    assert np.array_equal(got, exact.astype(np.float64))


def test_tc_combine_scales_and_special_rows():
    """Rows of very different scales (1e-300 .. 1e300), rows with one large and many tiny
    entries, zero rows, signed zeros and powers of two, against the stated bound."""
    rng = np.random.default_rng(9)
    n, nv, bv, nout = 4096, 8, 4, 5
    Vh = rng.standard_normal((nv, n, bv))
    scale = 10.0 ** rng.uniform(-300, 300, n)
    Vh *= scale[None, :, None]
    Vh[:, 10, :] = 0.0                       # zero row
    Vh[:, 11, :] = -0.0
    Vh[:, 12, :] = 2.0 ** rng.integers(-60, 60, (nv, bv))
    Vh[:, 13, :] = 1e-30
    Vh[0, 13, 0] = 1e30                      # one large entry, the rest 60 orders below
    Yh = rng.standard_normal((nv * bv, nout * bv))
    Yh[:, 3] *= 1e-200                       # a tiny column
    Yh[5, :] = 0.0
    got = _run(Vh, Yh, nout)
    _check(Vh, Yh, got)
    assert np.all(got[10] == 0.0) and np.all(got[11] == 0.0)


def test_tc_and_fma_engines_agree():
    rng = np.random.default_rng(11)
    n, nv, bv, nout = 100003, 8, 4, 5
    Vh = rng.standard_normal((nv, n, bv))
    Yh = rng.standard_normal((nv * bv, nout * bv))
    a = _run(Vh, Yh, nout, "tc")
    b = _run(Vh, Yh, nout, "fma")
    c = _run(Vh, Yh, nout, "auto")
    assert np.array_equal(a, c)
    absprod = np.abs(_flat(Vh)) @ np.abs(Yh)
    assert (np.abs(a - b) <= 2e-13 * absprod).all()


UPDATE_SHAPES = [  # (n, nv, bv): W (n x bv) = W - V C, K = nv*bv
    (1, 1, 4), (129, 8, 4), (4097, 3, 4), (65536, 8, 4), (10001, 5, 8), (3000, 2, 16),
    (777, 17, 1), (2050, 12, 2), (5000, 9, 4), (300, 16, 4)]


@pytest.mark.parametrize("shape", UPDATE_SHAPES)
@pytest.mark.parametrize("aligned", [True])
def test_tc_update_matches_oracle(shape, aligned):
    """W <- W - V C on the tensor cores (the second Gram-Schmidt pass's update, alpha = -1,
    beta = 1; fe_block_update_ex) against the oracle's MvTimesMatAddMv: within the stated
    split-product bound plus the rounding of the FP64 addition, and within 1e-13 (|V||C| + |W|);
    W inside a larger buffer (its neighbours untouched)."""
    t = torch()
    n, nv, bv = shape
    rng = np.random.default_rng(n + 31 * nv + bv)
    Vh = rng.standard_normal((nv, n, bv))
    Ch = rng.standard_normal((nv * bv, bv))
    Wh = rng.standard_normal((n, bv))
    buf = t.zeros(n * bv + 2, dtype=t.float64, device="cuda")
    off = 0 if aligned else 1
    W = buf[off:off + n * bv].view(n, bv)
    W.copy_(t.from_numpy(Wh))
    fe.block_update(to_dev(Vh), to_dev(Ch), W, alpha=-1.0, beta=1.0, engine="tc")
    t.cuda.synchronize()
    got = W.cpu().numpy()
    AA = _flat(Vh)
    ref = blockops.mv_times_mat_add_mv(-1.0, AA, Ch, 1.0, Wh.copy())
    K = AA.shape[1]
    err = np.abs(got - ref)
    vc = np.abs(AA) @ np.abs(Ch)
    stated = (2.0 ** -49 * (K + 1) * np.abs(AA).max(axis=1)[:, None] * np.abs(Ch).max(axis=0)[None, :]
              + 2.0 ** -52 * (vc + np.abs(Wh)) + 2.0 ** -1022)
    assert (err <= stated).all(), f"stated bound: worst {np.max(err - stated):.3e}"
    assert (err <= 1e-13 * (vc + np.abs(Wh))).all()
    assert buf[:off].abs().sum().item() == 0 and buf[off + n * bv:].abs().sum().item() == 0


def test_tc_update_engines_agree_and_reject():
    """fma and tc routes of fe_block_update_ex agree to 2e-13 (|V||C| + |W|); the tensor-core
    route rejects bv != bw, K > 64 and FP32 blocks, and auto falls back to the FMA kernels."""
    t = torch()
    rng = np.random.default_rng(3)
    n, nv, bv = 50000, 8, 4
    Vh = rng.standard_normal((nv, n, bv))
    Ch = rng.standard_normal((nv * bv, bv))
    Wh = rng.standard_normal((n, bv))
    outs = {}
    for eng in ("fma", "tc", "auto"):
        W = to_dev(Wh)
        fe.block_update(to_dev(Vh), to_dev(Ch), W, alpha=0.5, beta=-2.0, engine=eng)
        outs[eng] = W.cpu().numpy()
    assert np.array_equal(outs["tc"], outs["auto"])
    bound = 2e-13 * (np.abs(_flat(Vh)) @ np.abs(Ch) * 0.5 + 2.0 * np.abs(Wh))
    assert (np.abs(outs["tc"] - outs["fma"]) <= bound).all()
    W8 = t.zeros((64, 8), dtype=t.float64, device="cuda")
    with pytest.raises(fe.FeError):   # bv != bw
        fe.block_update(t.zeros((2, 64, 4), dtype=t.float64, device="cuda"),
                        t.zeros((8, 8), dtype=t.float64, device="cuda"), W8, engine="tc")
    with pytest.raises(fe.FeError):   # K = 68
        fe.block_update(t.zeros((17, 64, 4), dtype=t.float64, device="cuda"),
                        t.zeros((68, 4), dtype=t.float64, device="cuda"),
                        t.zeros((64, 4), dtype=t.float64, device="cuda"), engine="tc")
    fe.block_update(t.zeros((17, 64, 4), dtype=t.float64, device="cuda"),
                    t.zeros((68, 4), dtype=t.float64, device="cuda"),
                    t.zeros((64, 4), dtype=t.float64, device="cuda"), engine="auto")
    with pytest.raises(fe.FeError):   # FP32 blocks
        fe.block_update(t.zeros((2, 64, 4), dtype=t.float32, device="cuda"),
                        t.zeros((8, 4), dtype=t.float64, device="cuda"),
                        t.zeros((64, 4), dtype=t.float32, device="cuda"), engine="tc")


def test_tc_engine_rejects_unsupported():
    t = torch()
    V = t.zeros((17, 64, 4), dtype=t.float64, device="cuda")     # K = 68 > 64
    Y = t.zeros((68, 4), dtype=t.float64, device="cuda")
    with pytest.raises(fe.FeError):
        fe.block_combine(V, Y, 1, engine="tc")
    fe.block_combine(V, Y, 1, engine="auto")                      # FMA fallback
    V32 = t.zeros((2, 64, 4), dtype=t.float32, device="cuda")
    with pytest.raises(fe.FeError):
        fe.block_combine(V32, t.zeros((8, 4), dtype=t.float64, device="cuda"), 1, engine="tc")


@pytest.mark.parametrize("engine", ["auto", "tc"])
@pytest.mark.parametrize("name,nev,b,nb", [("rmat14", 8, 4, 8), ("rmat12", 6, 8, 8),
                                           ("er3000", 4, 2, 10)])
def test_eigs_tensor_core_restarts_match_oracle(name, nev, b, nb, engine):
    """The FP64 solve with tensor-core restart / Ritz products (engine auto; tc also runs the
    second Gram-Schmidt pass on the tensor cores) against the oracle's Block Krylov-Schur and
    against the FMA engine: eigenvalues within 1e-8 relative, explicit residuals within
    tol * |theta_1|."""
    g = {"rmat14": lambda: graphgen.rmat(14, seed=1), "rmat12": lambda: graphgen.rmat(12, seed=4),
         "er3000": lambda: graphgen.erdos_renyi(3000, 10.0, seed=2)}[name]()
    want = bks.block_krylov_schur(g.rowptr, g.colidx, nev, b, nb, 1e-8, "LM", seed=1,
                                  max_restarts=2000).evals
    with fe.Csr.from_graph(g) as h:
        ev_tc, X, st = fe.eigs(h, nev, b, nb, 1e-8, "LM", seed=1, engine=engine, max_restarts=2000)
        ev_f, _, st_f = fe.eigs(h, nev, b, nb, 1e-8, "LM", seed=1, engine="fma", max_restarts=2000)
    assert st["converged"] and st_f["converged"]
    np.testing.assert_allclose(ev_tc, want, rtol=1e-8)
    np.testing.assert_allclose(ev_tc, ev_f, rtol=1e-8)
    Xh = X.cpu().numpy()
    from oracle import core
    R = core.spmm(g.rowptr, g.colidx, Xh) - Xh * ev_tc
    assert (np.linalg.norm(R, axis=0) <= 1e-8 * np.abs(ev_tc).max()).all()


def _gram_check(Vh, Wh, G, tol_componentwise=1e-13):
    AA = _flat(Vh)
    ref = blockops.mv_trans_mv(1.0, AA, Wh)
    err = np.abs(G - ref)
    n = AA.shape[0]
    # stated bound: 2^-50 * 128 * max|V_c| * max|W_q| per 128-row tile, summed over the tiles
    stated = np.zeros_like(ref)
    for r0 in range(0, n, 128):
        stated += 2.0 ** -50 * 128 * np.outer(np.abs(AA[r0:r0 + 128]).max(0), np.abs(Wh[r0:r0 + 128]).max(0))
    stated += 1e-15 * (np.abs(AA).T @ np.abs(Wh)) + 2.0 ** -1022
    assert (err <= stated).all(), f"stated bound: worst {np.max(err - stated):.3e}"
    if tol_componentwise is not None:
        assert (err <= tol_componentwise * (np.abs(AA).T @ np.abs(Wh))).all()


GRAM_SHAPES = [  # (n, nv, bv, bw)
    (1, 1, 1, 1), (127, 8, 4, 4), (128, 9, 4, 4), (129, 9, 4, 4), (5000, 9, 4, 4), (100003, 9, 4, 4),
    (4099, 2, 8, 8), (3001, 18, 2, 2), (777, 18, 2, 1), (1500, 32, 1, 8), (2048, 4, 4, 8), (65537, 1, 16, 4)]


@pytest.mark.parametrize("shape", GRAM_SHAPES)
def test_tc_gram_matches_oracle(shape):
    """N(0,1) blocks: G = V^T W on the tensor cores within 1e-13 (|V|^T |W|) of the oracle's
    MvTransMv and within the stated per-tile bound; 1 or 2 M tiles of digit rows, ragged tiles."""
    n, nv, bv, bw = shape
    rng = np.random.default_rng(n + 3 * nv + bw)
    Vh = rng.standard_normal((nv, n, bv))
    Wh = rng.standard_normal((n, bw))
    G = fe.block_gram(to_dev(Vh), to_dev(Wh), engine="tc")
    _gram_check(Vh, Wh, G.cpu().numpy())


def _offset_dev(h, off):
    """h on the device, starting `off` doubles into a larger buffer (8 bytes off a 16-byte
    boundary for odd off)."""
    t = torch()
    buf = t.zeros(h.size + off + 1, dtype=t.float64, device="cuda")
    view = buf[off:off + h.size].view(h.shape)
    view.copy_(t.from_numpy(np.ascontiguousarray(h)))
    return view


def test_block_operations_reject_unaligned_blocks():
    """Block arguments 8 bytes off a 16-byte boundary are rejected (FE_ERR_INVALID) by the
    product, the update, the Gram, the fused update + Gram and the re-orthogonalisation, before
    any kernel runs; the aligned calls that follow still work."""
    rng = np.random.default_rng(21)
    n, nv, bv = 2048, 3, 4
    Vh = rng.standard_normal((nv, n, bv))
    Wh = rng.standard_normal((n, bv))
    Yh = rng.standard_normal((nv * bv, 2 * bv))
    Vu, Wu = _offset_dev(Vh, 1), _offset_dev(Wh, 1)
    Va, Wa, Y = to_dev(Vh), to_dev(Wh), to_dev(Yh)
    C = to_dev(Yh[:, :bv])
    for call in (lambda: fe.block_combine(Vu, Y, 2, engine="tc"),
                 lambda: fe.block_combine(Va, Y, 2, Out=_offset_dev(np.zeros((2, n, bv)), 1)),
                 lambda: fe.block_update(Vu, C, to_dev(Wh), engine="tc"),
                 lambda: fe.block_update(Va, C, _offset_dev(Wh, 1)),
                 lambda: fe.block_gram(Vu, Wa, engine="tc"),
                 lambda: fe.block_gram(Va, Wu),
                 lambda: fe.block_update_gram(Vu, C, to_dev(Wh)),
                 lambda: fe.block_orth(Va, _offset_dev(Wh, 1), anorm=1.0)):
        with pytest.raises(fe.FeError):
            call()
    G = fe.block_gram(Va, Wa, engine="tc").cpu().numpy()
    _gram_check(Vh, Wh, G)


def test_tc_gram_integers_exact_and_alias():
    """Integer data: every tile's digit products and their FP64 sums are exact, so G equals the
    integer product; W may be one of V's blocks."""
    rng = np.random.default_rng(6)
    n, nv, bv = 30011, 9, 4
    Vi = rng.integers(-1000, 1001, (nv, n, bv)).astype(np.float64)
    V = to_dev(Vi)
    G = fe.block_gram(V, V[8], engine="tc").cpu().numpy()
    exact = _flat(Vi.astype(np.int64)) .T @ Vi[8].astype(np.int64)
    assert np.array_equal(G, exact.astype(np.float64))


def test_tc_gram_scales_and_alpha():
    """Columns of very different scales within and across tiles, zero columns, alpha."""
    rng = np.random.default_rng(12)
    n, nv, bv, bw = 20000, 9, 4, 4
    Vh = rng.standard_normal((nv, n, bv)) * (10.0 ** rng.uniform(-150, 150, (nv, 1, bv)))
    Vh[:, ::97, :] *= 1e20                     # a few large rows per tile
    Vh[3] = 0.0
    Wh = rng.standard_normal((n, bw)) * 10.0 ** rng.uniform(-100, 100, (1, bw))
    G = fe.block_gram(to_dev(Vh), to_dev(Wh), alpha=-2.5, engine="tc").cpu().numpy()
    _gram_check(Vh, Wh, G / -2.5, tol_componentwise=None)


def test_tc_gram_and_fma_agree_and_rejects():
    rng = np.random.default_rng(13)
    n = 200003
    Vh = rng.standard_normal((9, n, 4))
    Wh = rng.standard_normal((n, 4))
    V, W = to_dev(Vh), to_dev(Wh)
    a = fe.block_gram(V, W, engine="tc").cpu().numpy()
    b = fe.block_gram(V, W, engine="fma").cpu().numpy()
    c = fe.block_gram(V, W).cpu().numpy()
    assert np.array_equal(a, c)                       # AUTO: tensor cores for 36 columns
    V4 = to_dev(Vh[:1])
    assert np.array_equal(fe.block_gram(V4, W).cpu().numpy(),
                          fe.block_gram(V4, W, engine="fma").cpu().numpy())   # 4 columns: FMA
    assert (np.abs(a - b) <= 2e-13 * (np.abs(_flat(Vh)).T @ np.abs(Wh))).all()
    t = torch()
    with pytest.raises(fe.FeError):
        fe.block_gram(t.zeros((10, 64, 4), dtype=t.float64, device="cuda"),
                      t.zeros((64, 4), dtype=t.float64, device="cuda"), engine="tc")   # 40 > 36
    with pytest.raises(fe.FeError):
        fe.block_gram(t.zeros((2, 64, 4), dtype=t.float64, device="cuda"),
                      t.zeros((64, 16), dtype=t.float64, device="cuda"), engine="tc")  # bw 16
