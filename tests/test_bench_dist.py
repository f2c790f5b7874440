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


def _bench(args, env=None, timeout=300):
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    e = dict(os.environ, **(env or {}))
    r = subprocess.run([sys.executable, *args], cwd=root, env=e, capture_output=True, text=True, timeout=timeout)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    return [json.loads(l) for l in lines]


def test_reference_arm_json_line():
    """bench.py --impl reference times the oracle on the host and prints one JSON line with the contract's keys."""
    (line,) = _bench(["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"])
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["steps"] == 1 and line["warmup"] == 3 and line["n_gpus"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"].startswith("1024x1024 cells, S16")


def test_reference_arm_rank0_only_under_torchrun():
    """Under torchrun with two ranks only rank 0 runs the oracle and prints; the other exits cleanly."""
    port = _free_port()
    lines = _bench(["-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
                    "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference", "--gpus", "2",
                    "--steps", "1", "--warmup", "3"], timeout=600)
    assert len(lines) == 1 and lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2
