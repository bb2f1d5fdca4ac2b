"""The multi-GPU path of bench.py on CPU: ranks are independent replicas and
the only collective is the max-over-ranks of the timed region (gloo,
world_size 2, 127.0.0.1)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    local_ms = 1000.0 * (rank + 1)           # rank 1 is the slow replica
    ms_max, value = bench.replica_throughput(local_ms, steps=5, ws=ws)
    q.put((rank, ms_max, value, bench.dist_info()))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, value, info in res:
        assert ms_max == 2000.0                      # slowest rank
        assert value == pytest.approx(2 * 5 / 2.0)   # all catalogs over the slowest time
        assert info == (2, rank, rank)
