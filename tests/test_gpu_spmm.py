"""GPU parity: fe_spmm against the oracle's plain-definition SpMM (Section 3.3).

Tolerances (the SpMM accuracy requirement of 1e-6 relative, read per entry against A|X|, the condition
number of a sum): FP64 |Y - Y*| <= 1e-13 (A|X|), FP32 <= 1e-6 (A|X|) with Y* the FP64 sum of
the same FP32 inputs.  A 1 = degree must be exact in either precision.  Inputs of one sign
(where rounding errors of a plain in-order sum do not cancel) are checked against the FP32
kernel's stated worst case, 9 * 2^-24 (A|X|).
"""
import numpy as np
import pytest

import graphgen
import paper_1602_01421_gb300 as fe
from tests.gpu_util import assert_spmm_close, to_dev, torch

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-6, "f64": 1e-13}
# the FP32 kernel's worst case per entry (compensated lane sums, <= 5 tree levels, one rounding
# of a split hub row's FP64 sum), in units of A|X|
F32_BOUND = 9 * 2.0 ** -24
# all-equal entries: a plain in-order FP32 sum of 127 (69) copies of this value is off by 1.47e-6
# (1.05e-6) of the exact sum (found by scanning 20000 values in [1, 2) with numpy float32 sums)
ADVERSARIAL_C = np.float32(1.9397392272949219)


def one_signed_block(kind, n, b, seed):
    """U[0,1), U[1,2) or the constant ADVERSARIAL_C, FP32, n x b."""
    if kind == "const":
        return np.full((n, b), ADVERSARIAL_C, dtype=np.float32)
    lo = 0.0 if kind == "u01" else 1.0
    return (lo + graphgen.uniform_block(n, b, seed=seed)).astype(np.float32)


def plain_sum_error(g, X, rows):
    """Largest |in-order FP32 sum - exact| / A|X| over `rows` (what a kernel summing each row
    in order, uncompensated, would get) -- shows that an input can catch such a kernel."""
    worst = 0.0
    for i in rows:
        cols = g.colidx[g.rowptr[i]:g.rowptr[i + 1]]
        if len(cols) == 0:
            continue
        s = np.zeros(X.shape[1], dtype=np.float32)
        for c in cols:
            s = (s + X[c]).astype(np.float32)
        exact = X[cols].astype(np.float64).sum(0)
        worst = max(worst, float((np.abs(s - exact) / np.abs(X[cols]).astype(np.float64).sum(0)).max()))
    return worst
NP = {"f32": np.float32, "f64": np.float64}

GRAPHS = {
    "rmat12": lambda: graphgen.rmat(12, seed=3),
    "rmat14": lambda: graphgen.rmat(14, seed=1),
    "rmat13-noperm": lambda: graphgen.rmat(13, seed=2, permute=False),
    "star9000": lambda: graphgen.star(9000),              # one hub split into 3 chunks
    "complete70": lambda: graphgen.complete(70),          # all rows in one slice bucket (deg 69)
    "complete128": lambda: graphgen.complete(128),        # slice rows of degree 127
    "complete300": lambda: graphgen.complete(300),        # all rows warp tasks (deg 299)
    "cycle1001": lambda: graphgen.cycle(1001),            # all rows tail (deg 2), ragged slice
    "er3000": lambda: graphgen.erdos_renyi(3000, 12.0, seed=5),
    "union-isolated": lambda: graphgen.disjoint_union(graphgen.star(5000), graphgen.path(33),
                                                      graphgen.from_edges(77, [], [], "iso77")),
}


@pytest.fixture(scope="module")
def graphs():
    return {k: v() for k, v in GRAPHS.items()}


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("b", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_spmm_parity(graphs, name, b, prec):
    g = graphs[name]
    X = graphgen.normal_block(g.n, b, seed=100 + b, dtype=NP[prec])
    with fe.Csr.from_graph(g) as h:
        Y = fe.spmm(h, to_dev(X)).cpu().numpy()
    assert_spmm_close(g, X, Y, TOL[prec])


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("knobs", [dict(tail_max=1, hub_min=8, hub_chunk=8),
                                   dict(tail_max=32, hub_min=40, hub_chunk=64),
                                   dict(tail_max=4, hub_min=64, hub_chunk=4096),
                                   dict(tail_max=128, hub_min=200, hub_chunk=100)])
def test_spmm_parity_all_paths_small(prec, knobs):
    """Tiny thresholds push most rows through the hub split and the partial reduce, with plain
    and with packed column indices."""
    g = graphgen.rmat(13, seed=9)
    for fmt in ("plain", "packed"):
        for b in (1, 4, 16):
            X = graphgen.normal_block(g.n, b, seed=b, dtype=NP[prec])
            with fe.Csr.from_graph(g, index_format=fmt, **knobs) as h:
                info = h.info()
                Y = fe.spmm(h, to_dev(X)).cpu().numpy()
            assert info["rows_hub"] > 0
            assert_spmm_close(g, X, Y, TOL[prec])


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("tail_max", [64, 128])
def test_spmm_parity_wide_tail(graphs, prec, tail_max):
    """Rows up to degree 64 / 128 in the thread-per-row slices (exact-degree buckets)."""
    for name in ("rmat14", "complete70", "er3000"):
        g = graphs[name]
        for b in (1, 4, 8, 16):
            X = graphgen.normal_block(g.n, b, seed=b + 7, dtype=NP[prec])
            with fe.Csr.from_graph(g, tail_max=tail_max) as h:
                info = h.info()
                Y = fe.spmm(h, to_dev(X)).cpu().numpy()
            deg = g.degrees()
            assert info["rows_tail"] == ((deg >= 1) & (deg <= tail_max)).sum()
            assert_spmm_close(g, X, Y, TOL[prec])


@pytest.mark.parametrize("prec,b", [("f32", 8), ("f32", 16), ("f64", 4), ("f64", 8), ("f64", 16)])
def test_spmm_parity_16_byte_aligned_blocks(graphs, prec, b):
    """X and Y 16-byte but not 32-byte aligned: the 16-byte gather path (32-byte rows are
    otherwise gathered with one 256-bit load per lane)."""
    t = torch()
    g = graphs["rmat14"]
    dt = t.float32 if prec == "f32" else t.float64
    shift = 16 // (4 if prec == "f32" else 8)
    X = graphgen.normal_block(g.n, b, seed=3, dtype=NP[prec])
    xbuf = t.zeros(g.n * b + 64, dtype=dt, device="cuda")
    ybuf = t.zeros(g.n * b + 64, dtype=dt, device="cuda")
    assert xbuf.data_ptr() % 32 == 0
    xv = xbuf[shift:shift + g.n * b].view(g.n, b)
    yv = ybuf[shift:shift + g.n * b].view(g.n, b)
    assert xv.data_ptr() % 32 == 16
    xv.copy_(to_dev(X))
    with fe.Csr.from_graph(g, tail_max=64) as h:
        fe.spmm(h, xv, yv)
        Y16 = yv.cpu().numpy()
        Y32 = fe.spmm(h, to_dev(X)).cpu().numpy()
    assert_spmm_close(g, X, Y16, TOL[prec])
    assert_spmm_close(g, X, Y32, TOL[prec])


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("name", ["rmat14", "rmat13-noperm", "star9000", "complete300", "er3000",
                                  "union-isolated"])
def test_spmm_parity_packed_index(graphs, prec, name):
    """Task rows' columns as bit-packed gaps (index_format packed): same results as the oracle,
    fewer index bytes than the plain plan."""
    g = graphs[name]
    with fe.Csr.from_graph(g, index_format="packed") as h, fe.Csr.from_graph(g, tail_max=16) as hp:
        info, info_plain = h.info(), hp.info()
        assert info["index_format"] == 2 and info_plain["index_format"] == 1
        assert info["tail_max"] == 16
        if info["rows_mid"] + info["rows_hub"] > 0:
            assert info["index_bytes"] < info_plain["index_bytes"]
        for b in (1, 2, 4, 8, 16):
            X = graphgen.normal_block(g.n, b, seed=b + 30, dtype=NP[prec])
            Y = fe.spmm(h, to_dev(X)).cpu().numpy()
            assert_spmm_close(g, X, Y, TOL[prec])
            # same column order and task split as the plain plan: identical results
            assert np.array_equal(Y, fe.spmm(hp, to_dev(X)).cpu().numpy())


@pytest.mark.parametrize("fmt", ["plain", "packed"])
def test_spmm_unsorted_rows_and_duplicates(fmt):
    """CSR rows in arbitrary order with repeated entries (A_ij = multiplicity); the packed
    plan sorts each row before taking gaps (gap 0 for a repeat)."""
    g = graphgen.rmat(12, seed=4)
    rng = np.random.default_rng(3)
    rows, cols = [], []
    for i in range(g.n):
        c = list(g.colidx[g.rowptr[i]:g.rowptr[i + 1]])
        c += [int(x) for x in rng.choice(c, size=min(len(c), 3), replace=False)] if c else []
        rng.shuffle(c)
        rows.append(len(c))
        cols.extend(c)
    rowptr = np.concatenate([[0], np.cumsum(rows)]).astype(np.int64)
    colidx = np.array(cols, dtype=np.int32)
    gu = graphgen.CSR(g.n, rowptr, colidx, "unsorted-dup")
    for prec in ("f32", "f64"):
        for b in (1, 4, 16):
            X = graphgen.normal_block(g.n, b, seed=b, dtype=NP[prec])
            with fe.Csr(rowptr, colidx, index_format=fmt, tail_max=8, hub_min=64, hub_chunk=48) as h:
                Y = fe.spmm(h, to_dev(X)).cpu().numpy()
            assert_spmm_close(gu, X, Y, TOL[prec])


@pytest.mark.parametrize("kind", ["u01", "u12", "const"])
@pytest.mark.parametrize("fmt", ["plain", "packed"])
@pytest.mark.parametrize("b", [1, 4, 16])
def test_spmm_f32_one_signed_inputs(graphs, kind, fmt, b):
    """FP32 with inputs of one sign (the rounding errors of a plain in-order sum then add up
    instead of cancelling): every entry within the stated worst case 9 * 2^-24 (A|X|), on
    graphs whose rows reach every path (slices up to degree 128, warp tasks, split hubs)."""
    for name in ("rmat14", "complete70", "complete128", "complete300", "star9000", "er3000"):
        g = graphs[name]
        X = one_signed_block(kind, g.n, b, seed=11 + b)
        with fe.Csr.from_graph(g, index_format=fmt) as h:
            Y = fe.spmm(h, to_dev(X)).cpu().numpy()
        ratio = assert_spmm_close(g, X, Y, F32_BOUND)
        assert ratio <= F32_BOUND
    if kind == "const" and fmt == "plain" and b == 1:
        # the constant input catches an uncompensated kernel: plain in-order sums of the
        # degree-69 and degree-127 rows of K70 and K128 miss the 1e-6 contract
        for name in ("complete70", "complete128"):
            g = graphs[name]
            assert plain_sum_error(g, one_signed_block("const", g.n, 1, 0), range(4)) > TOL["f32"]


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_ones_give_degrees_exactly(graphs, prec):
    t = torch()
    for name in ("rmat14", "star9000", "union-isolated"):
        g = graphs[name]
        with fe.Csr.from_graph(g) as h:
            for b in (1, 4, 16):
                X = t.ones((g.n, b), dtype=t.float32 if prec == "f32" else t.float64, device="cuda")
                Y = fe.spmm(h, X).cpu().numpy()
                assert np.array_equal(Y, np.repeat(g.degrees()[:, None], b, 1).astype(Y.dtype))


def test_empty_matrix_and_single_vertex():
    t = torch()
    for n in (1, 37):
        g = graphgen.from_edges(n, [], [], "empty")
        with fe.Csr.from_graph(g) as h:
            X = t.randn((n, 4), dtype=t.float64, device="cuda")
            Y = t.full_like(X, 7.0)
            fe.spmm(h, X, Y)
            assert t.count_nonzero(Y).item() == 0


def test_handle_info_bins(graphs):
    g = graphs["rmat14"]
    with fe.Csr.from_graph(g) as h:
        i = h.info()
    deg = g.degrees()
    assert i["n"] == g.n and i["nnz"] == g.nnz and i["max_degree"] == deg.max()
    assert i["rows_empty"] == (deg == 0).sum()
    assert i["rows_tail"] == ((deg >= 1) & (deg <= 128)).sum()
    assert i["rows_mid"] == ((deg > 128) & (deg <= 4096)).sum()
    assert i["rows_empty"] + i["rows_tail"] + i["rows_mid"] + i["rows_hub"] == g.n


def test_spmm_rejects_bad_arguments(graphs):
    t = torch()
    g = graphs["cycle1001"]
    with fe.Csr.from_graph(g) as h:
        X = t.zeros((g.n, 3), dtype=t.float64, device="cuda")
        with pytest.raises(fe.FeError):
            fe.spmm(h, X)                                  # b = 3 unsupported
        X = t.zeros((g.n, 4), dtype=t.float64, device="cuda")
        with pytest.raises(fe.FeError):
            fe.spmm(h, X, X)                               # in place
        big = t.zeros((2 * g.n * 4 + 2,), dtype=t.float64, device="cuda")
        lib = fe.load()                                    # misaligned (8-byte offset)
        rc = lib.fe_spmm(h.handle, big[1:].data_ptr(), big[g.n * 4 + 1:].data_ptr(), 4, 1)
        assert rc == -1 and b"aligned" in lib.fe_last_error()


@pytest.mark.slow
@pytest.mark.parametrize("prec,b", [("f32", 4), ("f64", 4), ("f32", 16), ("f64", 1)])
def test_spmm_full_size_sampled_rows(prec, b):
    """R-MAT scale 22 (the benchmark graph), in the benchmark's launch configuration; checked
    on 20000 random rows plus every hub row and the 2000 highest-degree rows."""
    g = graphgen.rmat(22, seed=1)
    X = graphgen.normal_block(g.n, b, seed=7, dtype=NP[prec])
    with fe.Csr.from_graph(g) as h:
        Y = fe.spmm(h, to_dev(X)).cpu().numpy()
    deg = g.degrees()
    rng = np.random.default_rng(0)
    rows = np.unique(np.concatenate([rng.integers(0, g.n, 20000), np.argsort(-deg)[:2000],
                                     np.nonzero(deg > 4096)[0]]))
    assert_spmm_close(g, X, Y, TOL[prec], rows=rows)
    # ones: exact degrees everywhere
    t = torch()
    with fe.Csr.from_graph(g) as h:
        ones = t.ones((g.n, b), dtype=t.float32 if prec == "f32" else t.float64, device="cuda")
        Yd = fe.spmm(h, ones)[:, 0].cpu().numpy()
    assert np.array_equal(Yd, deg.astype(Yd.dtype))


@pytest.mark.slow
@pytest.mark.parametrize("fmt", ["plain", "packed"])
@pytest.mark.parametrize("kind", ["u12", "const"])
def test_spmm_f32_one_signed_full_size(fmt, kind):
    """R-MAT scale 22, FP32 b in {1, 4, 16}, inputs of one sign: every row of degree 64..128
    (the longest thread-per-row sums of the default plan; warp tasks in the packed plan), every
    hub row and the 2000 highest-degree rows, within 9 * 2^-24 (A|X|)."""
    g = graphgen.rmat(22, seed=1)
    deg = g.degrees()
    rows = np.unique(np.concatenate([np.nonzero((deg >= 64) & (deg <= 128))[0],
                                     np.argsort(-deg)[:2000], np.nonzero(deg > 4096)[0]]))
    with fe.Csr.from_graph(g, index_format=fmt) as h:
        for b in (1, 4, 16):
            X = one_signed_block(kind, g.n, b, seed=5 + b)
            Y = fe.spmm(h, to_dev(X)).cpu().numpy()
            assert assert_spmm_close(g, X, Y, F32_BOUND, rows=rows) <= F32_BOUND


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_spmm_l2_window_same_results(graphs, prec):
    """An L2 access-policy window on X (l2_persist) changes only cache policy: identical results."""
    g = graphs["rmat14"]
    for b in (1, 4, 16):
        X = to_dev(graphgen.normal_block(g.n, b, seed=b, dtype=NP[prec]))
        with fe.Csr.from_graph(g) as h, fe.Csr.from_graph(g, l2_persist=True) as hl:
            assert np.array_equal(fe.spmm(h, X).cpu().numpy(), fe.spmm(hl, X).cpu().numpy())
