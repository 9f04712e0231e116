"""Row partition for a multi-GPU layout (fe_partition_rows, fe_partition_local, the dist module):
host logic on the CPU, and the row-partitioned SpMM + Gram steps over 2 gloo ranks, each rank
applying the oracle's SpMM to its local CSR, checked against the oracle on the whole matrix."""
import os
import socket

import numpy as np
import pytest

import graphgen
from paper_1602_01421_gb300 import dist as fdist

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("g", [graphgen.rmat(12, seed=2), graphgen.star(3000), graphgen.path(17),
                               graphgen.rmat(10, seed=5, permute=False)], ids=lambda g: g.name)
@pytest.mark.parametrize("nparts", [1, 2, 3, 8])
def test_partition_rows_balanced_and_covering(g, nparts):
    b = fdist.partition_rows(g.rowptr, nparts)
    assert b[0] == 0 and b[-1] == g.n and np.all(np.diff(b) >= 0)
    cost = g.rowptr[1:] - g.rowptr[:-1] + 1                     # non-zeros + 1 per row
    part_cost = np.array([cost[b[p]:b[p + 1]].sum() for p in range(nparts)])
    assert part_cost.sum() == cost.sum()
    assert part_cost.max() <= cost.sum() / nparts + cost.max()


def test_partition_local_csr_and_halo():
    g = graphgen.rmat(11, seed=3)
    for nparts in (2, 5):
        seen = 0
        for rank in range(nparts):
            p = fdist.RowPart(g.rowptr, g.colidx, nparts, rank)
            assert p.rowptr[0] == 0 and p.rowptr.shape[0] == p.rows + 1
            lo, hi = g.rowptr[p.r0], g.rowptr[p.r1]
            assert np.array_equal(p.rowptr, g.rowptr[p.r0:p.r1 + 1] - lo)
            assert np.array_equal(p.colidx, g.colidx[lo:hi])
            ext = np.unique(g.colidx[lo:hi][(g.colidx[lo:hi] < p.r0) | (g.colidx[lo:hi] >= p.r1)])
            assert np.array_equal(p.halo, ext)
            own = p.halo_owner()
            assert np.all(own != rank) and np.all((p.bounds[own] <= p.halo) & (p.halo < p.bounds[own + 1]))
            seen += p.rows
        assert seen == g.n


def test_partition_rejects_bad_arguments():
    from paper_1602_01421_gb300 import FeError
    with pytest.raises(FeError):
        fdist.partition_rows(np.array([0, 2, 1], dtype=np.int64), 2)      # decreasing rowptr
    with pytest.raises(FeError):
        fdist.partition_rows(np.array([0, 1], dtype=np.int64), 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import graphgen
    from oracle import core
    from paper_1602_01421_gb300 import dist as fdist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        g = graphgen.rmat(11, seed=7)
        part = fdist.RowPart(g.rowptr, g.colidx, ws, rank)
        X = graphgen.normal_block(g.n, 4, seed=3)                  # the global block (seeded)
        Xi = np.random.default_rng(4).integers(-50, 51, (g.n, 4)).astype(np.float64)
        V = graphgen.normal_block(g.n, 12, seed=5)                 # three 4-column basis blocks
        out = {}
        for name, Xg in (("normal", X), ("integer", Xi)):
            x_local = torch.from_numpy(Xg[part.r0:part.r1].copy())
            # the oracle's SpMM on the local rows (global column ids; rows >= rows() empty)
            rp = np.concatenate([part.rowptr, np.full(g.n - part.rows, part.rowptr[-1])])

            def spmm_local(x_full):
                return torch.from_numpy(core.spmm(rp, part.colidx, x_full.numpy())[:part.rows])

            x_full = fdist.allgather_rows(x_local, part, dist)
            y_local = fdist.spmm_step(part, x_local, spmm_local, dist)
            # halo suffices: X rows that are neither local nor in the halo can be anything
            xh = x_full.clone()
            keep = np.zeros(g.n, bool)
            keep[part.r0:part.r1] = True
            keep[part.halo] = True
            xh[torch.from_numpy(~keep)] = float("nan")
            y_halo = spmm_local(xh)
            v_local = torch.from_numpy(V[part.r0:part.r1].copy())
            G = fdist.gram_step(v_local, y_local, dist)             # V^T (A X)
            S = fdist.gram_step(y_local, y_local, dist)             # (A X)^T (A X)
            out[name] = (np.array_equal(x_full.numpy(), Xg), y_local.numpy(), y_halo.numpy(),
                         G.numpy(), S.numpy())
        q.put((rank, part.r0, part.r1, out))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_row_partitioned_spmm_and_gram_two_gloo_ranks():
    """2 ranks: all-gathered X equals the global block; each rank's rows of A X equal the global
    oracle's rows exactly (same row sums in the same order) and do not depend on X rows outside
    the part and its halo; the all-reduced V^T (A X) and (A X)^T (A X) match the global oracle
    (exactly for integer data)."""
    import torch.multiprocessing as mp
    from oracle import core
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    g = graphgen.rmat(11, seed=7)
    V = graphgen.normal_block(g.n, 12, seed=5)
    inputs = {"normal": graphgen.normal_block(g.n, 4, seed=3),
              "integer": np.random.default_rng(4).integers(-50, 51, (g.n, 4)).astype(np.float64)}
    assert res[0][1] == 0 and res[0][2] == res[1][1] and res[1][2] == g.n
    for name, Xg in inputs.items():
        Y = core.spmm(g.rowptr, g.colidx, Xg)
        G = V.T @ Y
        S = Y.T @ Y
        for rank, r0, r1, out in res:
            same_x, y_local, y_halo, Gp, Sp = out[name]
            assert same_x
            assert np.array_equal(y_local, Y[r0:r1])
            assert np.array_equal(y_halo, Y[r0:r1])
            if name == "integer":
                assert np.array_equal(Sp, S)
            bound = 1e-13 * (np.abs(V).T @ np.abs(Y))
            assert np.all(np.abs(Gp - G) <= bound)
            assert np.all(np.abs(Sp - S) <= 1e-13 * (np.abs(Y).T @ np.abs(Y)))
