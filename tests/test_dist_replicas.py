"""The N > 1 bench path (replicas: every rank solves its own copy; value = all ranks' solves over
the slowest rank's time), exercised with 2 gloo ranks on the CPU."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    local_ms = 1000.0 * (rank + 1)            # rank 1 is the slowest: 2000 ms for 4 steps
    value, ms, n = bench.replica_aggregate(local_ms, 4, dist, device="cpu")
    q.put((rank, value, ms, n))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, ms, n in res:
        assert n == 2 and ms == 2000.0
        assert abs(value - 2 * 4 / 2.0) < 1e-12      # 8 solves in 2 s on the job clock


def test_replica_aggregate_single_process():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    value, ms, n = bench.replica_aggregate(500.0, 5, None)
    assert (value, ms, n) == (10.0, 500.0, 1)
