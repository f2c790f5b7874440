"""Multi-rank host logic of bench.py on the CPU (gloo, world size 2): each rank is an independent replica;
the job's time is the slowest rank's and its work the sum over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms, upd = bench.aggregate(100.0 + 50.0 * rank, 1000 * (rank + 1), dist)
    dist.barrier()
    q.put((rank, ms, upd))
    dist.destroy_process_group()


def test_aggregate_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, upd in out:
        assert ms == 150.0 and upd == 3000.0


def test_aggregate_single_process():
    import bench
    assert bench.aggregate(12.5, 7, None) == (12.5, 7)
