"""Row-partitioned SpMM and Gram steps over torch.distributed (one rank per GPU).

The paper's solver runs on one machine (Section 3); over several GPUs the method shards by rows
(a part owns a contiguous row range of A and of every n x b block) with two exchanges:

  * SpMM (Section 3.3): a part multiplies its row block of A, which references X rows of other
    parts, so X is all-gathered (or only the "halo" rows its columns reference are fetched);
  * Gram products (MvTransMv, Table 1): V^T W is the sum of the parts' partial products, an
    all-reduce of the small (k x b) result; the same holds for W^T W in CholQR.

The row partition and the local CSR come from the library (fe_partition_rows,
fe_partition_local); the SpMM itself is the caller's function of (local CSR, gathered X), so the
same step runs with the library's kernels on a GPU (a rectangular handle, fe_csr_opts.ncols) or
with any other implementation.
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._lib import check, load


def partition_rows(rowptr: np.ndarray, nparts: int) -> np.ndarray:
    """Row boundaries (nparts + 1) of near-equal cost (non-zeros + rows) per part."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    n = rowptr.shape[0] - 1
    out = np.zeros(nparts + 1, dtype=np.int64)
    check(load().fe_partition_rows(n, rowptr.ctypes.data_as(ctypes.c_void_p), int(nparts),
                                   out.ctypes.data_as(ctypes.c_void_p)))
    return out


class RowPart:
    """Part `rank` of a row partition: rows [r0, r1), local CSR with global column ids, halo."""

    def __init__(self, rowptr: np.ndarray, colidx: np.ndarray, nparts: int, rank: int):
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        colidx = np.ascontiguousarray(colidx, dtype=np.int32)
        self.n = int(rowptr.shape[0] - 1)
        self.nparts, self.rank = int(nparts), int(rank)
        self.bounds = partition_rows(rowptr, nparts)
        self.r0, self.r1 = int(self.bounds[rank]), int(self.bounds[rank + 1])
        nnz = int(rowptr[self.r1] - rowptr[self.r0])
        self.rowptr = np.zeros(self.r1 - self.r0 + 1, dtype=np.int64)
        self.colidx = np.zeros(max(nnz, 1), dtype=np.int32)
        halo = np.zeros(max(nnz, 1), dtype=np.int32)
        nh = ctypes.c_int64(0)
        check(load().fe_partition_local(self.n, rowptr.ctypes.data_as(ctypes.c_void_p),
                                        colidx.ctypes.data_as(ctypes.c_void_p), self.r0, self.r1,
                                        self.rowptr.ctypes.data_as(ctypes.c_void_p),
                                        self.colidx.ctypes.data_as(ctypes.c_void_p),
                                        halo.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nh)))
        self.colidx = self.colidx[:nnz]
        self.halo = halo[:nh.value].copy()

    @property
    def rows(self) -> int:
        return self.r1 - self.r0

    def halo_owner(self) -> np.ndarray:
        """Owning part of every halo column."""
        return np.searchsorted(self.bounds, self.halo, side="right") - 1

    def csr(self, **kw):
        """Rectangular (rows x n) device handle of the local rows (GPU path)."""
        from . import Csr
        return Csr(self.rowptr, self.colidx, ncols=self.n, **kw)


def allgather_rows(x_local, part: RowPart, dist, group=None):
    """The full n x b block from every part's row block (torch.distributed all-gather; the row
    blocks are padded to the largest part)."""
    import torch
    sizes = np.diff(part.bounds)
    m = int(sizes.max())
    pad = torch.zeros((m,) + tuple(x_local.shape[1:]), dtype=x_local.dtype, device=x_local.device)
    pad[: x_local.shape[0]] = x_local
    bufs = [torch.empty_like(pad) for _ in range(part.nparts)]
    dist.all_gather(bufs, pad, group=group)
    return torch.cat([bufs[p][: int(sizes[p])] for p in range(part.nparts)], dim=0)


def allreduce_sum(t, dist, group=None):
    """Sum of the parts' partial results (Gram products V^T W, W^T W), in place."""
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def spmm_step(part: RowPart, x_local, spmm_local, dist, group=None):
    """Y rows [r0, r1) of A X: all-gather X, then the local row block's SpMM."""
    x_full = allgather_rows(x_local, part, dist, group)
    return spmm_local(x_full)


def gram_step(v_local, w_local, dist, group=None):
    """V^T W over all parts: the local (k x b) product, then an all-reduce."""
    g = v_local.transpose(0, 1).to(w_local.dtype) @ w_local
    return allreduce_sum(g.contiguous(), dist, group)
