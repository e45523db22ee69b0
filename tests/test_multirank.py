"""Multi-rank benchmark path on CPU (gloo, world size 2).

The benchmark runs one independent replica per rank (the update has no
exchange step to distribute); the job's throughput is the total of all
ranks' updates over the slowest rank's time.  This checks that reduction
with two gloo ranks on the CPU."""
import os

import pytest


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ups, el = bench.reduce_over_ranks(1000 * (rank + 1), 2.0 + rank)
    q.put((rank, ups, el))
    dist.destroy_process_group()


def test_replicas_reduce_to_total_over_slowest():
    mp = pytest.importorskip("torch.multiprocessing")
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in ps)
    for rank, ups, el in out:
        assert el == pytest.approx(3.0)
        assert ups == pytest.approx(3000 / 3.0)
