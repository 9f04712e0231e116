"""Helpers for the GPU parity tests (the CUDA path is compared with the CPU oracle)."""
import numpy as np

from oracle import core


def torch():
    import torch as t
    if not t.cuda.is_available():
        raise RuntimeError("GPU tests need CUDA")
    return t


def to_dev(a, dtype=None):
    t = torch()
    x = t.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        x = x.to(dtype)
    return x.cuda()


def spmm_bound(g, X64, rel):
    """rel * (A |X|): the condition-aware per-entry bound of the SpMM parity tests."""
    return rel * core.spmm(g.rowptr, g.colidx, np.abs(X64))


def assert_spmm_close(g, X, Y_gpu, rel, rows=None):
    """Y_gpu vs the oracle on the same X (float32 X is widened exactly)."""
    X64 = np.asarray(X, dtype=np.float64)
    if rows is None:
        ref = core.spmm(g.rowptr, g.colidx, X64)
        bound = spmm_bound(g, X64, rel)
        got = Y_gpu
    else:
        ref = core.spmm_rows(g.rowptr, g.colidx, X64, rows)
        bound = rel * core.spmm_rows(g.rowptr, g.colidx, np.abs(X64), rows)
        got = Y_gpu[rows]
    err = np.abs(got.astype(np.float64) - ref)
    bad = err > bound
    assert not bad.any(), (f"{bad.sum()} entries out of bound; worst err {err.max():.3e}, "
                           f"at bound {bound[np.unravel_index(np.argmax(err - bound), err.shape)]:.3e}")
    return float((err / np.maximum(bound / rel, 1e-300)).max())
