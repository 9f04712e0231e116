"""Semi-external SpMM (Section 3.3: sparse matrix streamed in panels while the dense blocks stay
in device memory) against the resident SpMM and the oracle."""
import ctypes

import numpy as np
import pytest

import graphgen
import paper_1602_01421_gb300 as fe
from tests.gpu_util import assert_spmm_close, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g16():
    return graphgen.rmat(16, seed=5)


@pytest.mark.parametrize("direct", [False, True])
@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("b", [1, 4, 16])
def test_semiext_equals_resident_and_oracle(g16, prec, b, direct):
    X = graphgen.normal_block(g16.n, b, seed=b, dtype=np.float32 if prec == "f32" else np.float64)
    Xd = to_dev(X)
    with fe.Csr.from_graph(g16, device_mem_cap_bytes=3 << 20, semi_direct=direct) as hs:
        info = hs.info()
        Ys = fe.spmm(hs, Xd).cpu().numpy()
    # semi-external handles default to packed indices and a small slice cutoff; the resident
    # handle takes the same plan shape
    assert info["index_format"] == 2 and 4 <= info["tail_max"] <= 16
    with fe.Csr.from_graph(g16, tail_max=info["tail_max"], index_format="packed") as hr:
        Yr = fe.spmm(hr, Xd).cpu().numpy()
    assert info["semi_external"] == 1 and info["panels"] > 2
    assert info["device_bytes"] <= 3 << 20
    assert np.array_equal(Ys, Yr)          # same per-row arithmetic, panel by panel
    assert_spmm_close(g16, X, Ys, 1e-6 if prec == "f32" else 1e-13)


def test_semiext_small_panels_and_hubs():
    g = graphgen.disjoint_union(graphgen.star(20000), graphgen.rmat(13, seed=1))
    X = graphgen.normal_block(g.n, 4, seed=2)
    with fe.Csr.from_graph(g, device_mem_cap_bytes=1 << 20, panel_nnz=20000, hub_min=1000,
                           hub_chunk=512) as hs:
        assert hs.info()["panels"] >= 10
        Y = fe.spmm(hs, to_dev(X)).cpu().numpy()
    assert_spmm_close(g, X, Y, 1e-13)


@pytest.mark.parametrize("direct", [False, True])
def test_semiext_eigs_matches_resident(direct):
    g = graphgen.rmat(14, seed=1)
    with fe.Csr.from_graph(g, device_mem_cap_bytes=1 << 20, semi_direct=direct) as hs:
        assert hs.info()["semi_external"] == 1
        tm = hs.info()["tail_max"]
        ev_s, X, st_s = fe.eigs(hs, 8, 4, 8, 1e-8, "LM", seed=1)
    with fe.Csr.from_graph(g, tail_max=tm, index_format="packed") as hr:
        ev_r, _, st_r = fe.eigs(hr, 8, 4, 8, 1e-8, "LM", seed=1)
    assert np.allclose(ev_s, ev_r, rtol=1e-12) and st_s["restarts"] == st_r["restarts"]


@pytest.mark.parametrize("fmt", ["plain", "packed"])
def test_semiext_index_formats_match_oracle(g16, fmt):
    """Both column-index formats streamed in panels; packed panels move fewer bytes."""
    X = graphgen.normal_block(g16.n, 4, seed=21)
    with fe.Csr.from_graph(g16, device_mem_cap_bytes=3 << 20, index_format=fmt) as hs:
        info = hs.info()
        Y = fe.spmm(hs, to_dev(X)).cpu().numpy()
    assert info["semi_external"] == 1 and info["index_format"] == (2 if fmt == "packed" else 1)
    if fmt == "packed":
        assert info["index_bytes"] < 0.8 * 4 * g16.nnz
    assert_spmm_close(g16, X, Y, 1e-13)


def test_cap_large_enough_stays_resident(g16):
    with fe.Csr.from_graph(g16, device_mem_cap_bytes=1 << 30) as h:
        assert h.info()["semi_external"] == 0


def test_cap_too_small_is_rejected(g16):
    with pytest.raises(fe.FeError) as e:
        fe.Csr.from_graph(g16, device_mem_cap_bytes=16 << 10)
    assert e.value.code == -1


def test_semiext_wait_bound_returns_timeout_then_result_completes():
    """A host-side wait bound that runs out returns FE_ERR_TIMEOUT while the GPU work goes on;
    after a device synchronisation the result is complete and correct."""
    t = torch()
    g = graphgen.rmat(21, seed=3)       # one SpMM of this size takes well over the 1 ms bound
    X = graphgen.normal_block(g.n, 16, seed=4)
    Xd = to_dev(X)
    Y = t.zeros_like(Xd)
    with fe.Csr.from_graph(g, device_mem_cap_bytes=64 << 20, panel_nnz=1 << 20,
                           copy_timeout_ms=1) as hs:
        fe._stream()
        lib = fe.load()
        rc = lib.fe_spmm(hs.handle, ctypes.c_void_p(Xd.data_ptr()), ctypes.c_void_p(Y.data_ptr()), 16, 1)
        assert rc == -5, lib.fe_last_error()
        assert b"not done" in lib.fe_last_error()
        t.cuda.synchronize()
        rows = np.unique(np.concatenate([np.random.default_rng(2).integers(0, g.n, 20000),
                                         np.argsort(-g.degrees())[:500]]))
        assert_spmm_close(g, X, Y.cpu().numpy(), 1e-13, rows=rows)


@pytest.mark.slow
def test_semiext_full_size_sampled_rows():
    """R-MAT scale 22 streamed in panels under a 256 MB cap (the bench's semi-external leg),
    checked on sampled rows plus every hub row, and A 1 = degree exactly."""
    t = torch()
    g = graphgen.rmat(22, seed=1)
    X = graphgen.normal_block(g.n, 4, seed=11, dtype=np.float32)
    with fe.Csr.from_graph(g, device_mem_cap_bytes=256 << 20) as hs:
        assert hs.info()["panels"] > 2
        Y = fe.spmm(hs, to_dev(X)).cpu().numpy()
        ones = t.ones((g.n, 1), dtype=t.float64, device="cuda")
        deg = fe.spmm(hs, ones)[:, 0].cpu().numpy()
    assert np.array_equal(deg, g.degrees().astype(np.float64))
    d = g.degrees()
    rows = np.unique(np.concatenate([np.random.default_rng(1).integers(0, g.n, 20000),
                                     np.nonzero(d > 4096)[0]]))
    assert_spmm_close(g, X, Y, 1e-6, rows=rows)
