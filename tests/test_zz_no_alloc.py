"""fe_block_gram_noalloc: the Gram product for callers that cannot allocate device memory
(their device memory is reserved by their own allocator, or they must avoid calls that can
synchronise the device).  Called through the C ABI and compared with fe_block_gram, the
allocating entry point, on two calls in a row.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import graphgen
import paper_1602_01421_gb300 as fe
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
