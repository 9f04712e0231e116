"""Row-partitioned SpMM on the GPU: each part of a row partition as a rectangular handle
(rows x n, global column ids; fe_csr_opts.ncols) runs the same SpMM kernels on the full X.
Parts are processed one after another on one GPU; the collectives of the multi-GPU step are
tested on CPU ranks (tests/test_partition.py)."""
import numpy as np
import pytest

import graphgen
import paper_1602_01421_gb300 as fe
from paper_1602_01421_gb300 import dist as fdist
from tests.gpu_util import assert_spmm_close, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("nparts", [2, 3, 7])
def test_partitioned_spmm_equals_global(prec, nparts):
    """Concatenated part results equal the single-handle SpMM bit for bit (every row keeps its
    degree class and summation order) and match the oracle."""
    g = graphgen.rmat(14, seed=1)
    dt = np.float32 if prec == "f32" else np.float64
    for b in (1, 4, 16):
        X = graphgen.normal_block(g.n, b, seed=b, dtype=dt)
        Xd = to_dev(X)
        with fe.Csr.from_graph(g) as h:
            Yg = fe.spmm(h, Xd).cpu().numpy()
        parts = []
        for rank in range(nparts):
            p = fdist.RowPart(g.rowptr, g.colidx, nparts, rank)
            with p.csr() as hp:
                info = hp.info()
                assert info["n"] == p.rows and info["ncols"] == g.n
                parts.append(fe.spmm(hp, Xd).cpu().numpy())
        Y = np.concatenate(parts)
        assert np.array_equal(Y, Yg)
        assert_spmm_close(g, X, Y, 1e-6 if prec == "f32" else 1e-13)


def test_rectangular_handle_rules():
    t = torch()
    g = graphgen.rmat(10, seed=2)
    p = fdist.RowPart(g.rowptr, g.colidx, 2, 0)
    with p.csr() as hp:
        with pytest.raises(fe.FeError):
            fe.eigs(hp, 2, 2, 4, 1e-8, "LM")                    # not square
    with pytest.raises(fe.FeError):
        fe.Csr(p.rowptr, p.colidx, ncols=g.n, transpose=True)  # rectangular + transpose
    with pytest.raises(fe.FeError):
        fe.Csr(p.rowptr, p.colidx, ncols=int(g.colidx.max()))  # a column >= ncols
