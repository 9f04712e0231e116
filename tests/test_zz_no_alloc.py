"""fe_block_gram_noalloc: the Gram product for callers that cannot allocate device memory
(their device memory is reserved by their own allocator, or they must avoid calls that can
synchronise the device).  Called through the C ABI and compared with fe_block_gram, the
allocating entry point, on two calls in a row, and with the oracle's MvTransMv (Table 1).
Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import graphgen
import paper_1602_01421_gb300 as fe
from oracle import blockops
from tests.gpu_util import to_dev, torch

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f64": 1e-13}   # the Gram tolerance of tests/test_gpu_blockops.py
NP = {"f32": np.float32, "f64": np.float64}


def _noalloc(lib, V, W, alpha, G):
    nv, n, bv = V.shape
    bw = W.shape[1]
    dt = 0 if V.dtype == torch().float32 else 1
    return lib.fe_block_gram_noalloc(ctypes.c_void_p(V.data_ptr()), n, nv, bv,
                                     ctypes.c_void_p(W.data_ptr()), bw, dt, float(alpha),
                                     ctypes.c_void_p(G.data_ptr()))


def _lib():
    lib = fe.load()
    f = lib.fe_block_gram_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_void_p]
    return lib


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_noalloc_gram_matches_allocating_gram_twice(prec):
    t = torch()
    lib = _lib()
    fe._stream()
    for call, (n, nv, bv, bw, seed) in enumerate([(300007, 9, 4, 4, 1), (123457, 3, 8, 8, 2)]):
        V = to_dev(graphgen.normal_block(nv * n, bv, seed=seed, dtype=NP[prec]).reshape(nv, n, bv))
        W = to_dev(graphgen.normal_block(n, bw, seed=seed + 10, dtype=NP[prec]))
        G = t.full((nv * bv, bw), float("nan"), dtype=t.float64, device="cuda")
        assert _noalloc(lib, V, W, 0.5, G) == 0, lib.fe_last_error()
        ref = fe.block_gram(V, W, alpha=0.5)
        t.cuda.synchronize()
        absprod = 0.5 * (V.abs().to(t.float64).permute(0, 2, 1).reshape(nv * bv, n)
                         @ W.abs().to(t.float64))
        err = (G - ref).abs()
        assert t.isfinite(G).all(), f"call {call}"
        assert bool((err <= TOL[prec] * absprod).all()), f"call {call}: max err {err.max().item()}"


def test_noalloc_gram_rejects_oversized_output():
    t = torch()
    lib = _lib()
    V = t.zeros((16, 64, 16), dtype=t.float64, device="cuda")   # 16*16*16 = 4096 > 2048
    W = t.zeros((64, 16), dtype=t.float64, device="cuda")
    G = t.zeros((256, 16), dtype=t.float64, device="cuda")
    assert _noalloc(lib, V, W, 1.0, G) == -1
    assert b"2048" in lib.fe_last_error()


def _oracle_check(V, W, alpha, G, tol):
    """G against the oracle's MvTransMv on the same inputs, per entry within
    tol * alpha * (|V|^T |W|)."""
    Vh = V.cpu().numpy().astype(np.float64)
    Wh = W.cpu().numpy().astype(np.float64)
    nv, n, bv = Vh.shape
    AA = Vh.transpose(1, 0, 2).reshape(n, nv * bv)   # column j*bv + p = block j's column p
    ref = blockops.mv_trans_mv(alpha, AA, Wh)
    bound = tol * abs(alpha) * (np.abs(AA).T @ np.abs(Wh))
    err = np.abs(G.cpu().numpy() - ref)
    assert (err <= bound).all(), f"max err {err.max():.3e}"


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("shape", [(8, 16, 16), (4, 16, 2), (32, 2, 16), (5, 1, 8)])
def test_noalloc_gram_matches_oracle_at_and_below_the_size_limit(prec, shape):
    """nv * bv * bw up to the 2048-entry limit: at the limit the static scratch holds 128 CTAs'
    partials, so the grid is cut to fit it; bv != bw gives non-square output tiles.  Two calls
    in a row on different inputs, each checked against the oracle and against fe_block_gram."""
    t = torch()
    lib = _lib()
    fe._stream()
    nv, bv, bw = shape
    for call, n in enumerate([200003, 65537]):
        V = to_dev(graphgen.normal_block(nv * n, bv, seed=40 + call, dtype=NP[prec]).reshape(nv, n, bv))
        W = to_dev(graphgen.normal_block(n, bw, seed=50 + call, dtype=NP[prec]))
        G = t.full((nv * bv, bw), float("nan"), dtype=t.float64, device="cuda")
        assert _noalloc(lib, V, W, -1.5, G) == 0, lib.fe_last_error()
        ref = fe.block_gram(V, W, alpha=-1.5)
        t.cuda.synchronize()
        assert t.isfinite(G).all(), f"call {call}"
        _oracle_check(V, W, -1.5, G, TOL[prec])
        absprod = 1.5 * (V.abs().to(t.float64).permute(0, 2, 1).reshape(nv * bv, n)
                         @ W.abs().to(t.float64))
        assert bool(((G - ref).abs() <= 2 * TOL[prec] * absprod).all()), f"call {call}"
