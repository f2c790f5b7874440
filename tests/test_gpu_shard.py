"""Angle sharding through the C ABI on one GPU.

(1) Sweeping every chunk of the partial sets with lmdg_sweep_shard and combining them with lmdg_sweep_combine gives
lmdg_sweep's result bit for bit, for every scheme and arithmetic, with chunks that hold several sets, one set or
none.  (2) Repeated applications, each chunk swept by its own context of the problem (what each GPU of a sharded
run holds), stay bitwise equal.  (3) The torch.distributed helper on a group of one rank.
"""
import numpy as np
import pytest

from tests.helpers import random_problem

pytestmark = pytest.mark.gpu


def _ctx(p, variant, **kw):
    from paper_1907_01027_gb300 import Context
    return Context(p, variant, **kw)


def _flags():
    from paper_1907_01027_gb300 import SWEEP_SOURCE, SWEEP_FP32, SWEEP_F32X2
    return {"fp64": 0, "fp64-src": SWEEP_SOURCE, "fp32": SWEEP_FP32, "fp32-src": SWEEP_FP32 | SWEEP_SOURCE,
            "f32x2-src": SWEEP_F32X2 | SWEEP_SOURCE}


@pytest.mark.parametrize("variant", ["std", "lm", "rlm", "p0"])
@pytest.mark.parametrize("mode", ["fp64", "fp64-src", "fp32", "fp32-src", "f32x2-src"])
@pytest.mark.parametrize("N,nshards", [(4, 2), (4, 7), (8, 3), (16, 5)])
def test_shard_sweeps_combine_to_the_sweep(variant, mode, N, nshards):
    import torch
    flags = _flags()[mode]
    p = random_problem(37, N, 0.7, 3, ny=45)
    ctx = _ctx(p, variant)
    x = torch.from_numpy(np.random.default_rng(1).standard_normal((p.nx, 4))).cuda()
    y_ref = ctx.sweep(x, flags=flags)
    sets, chunk, nbytes = ctx.shard_layout(nshards, flags)
    assert chunk == -(-sets // nshards) and nbytes % 8 == 0   # sets start 8-byte aligned (NR floats, NR even)
    parts = torch.empty(nshards * nbytes, dtype=torch.uint8, device="cuda")
    for r in reversed(range(nshards)):   # any order: each chunk is written by its own shard only
        ctx.sweep_shard(x, parts, r, nshards, flags)
    y = ctx.sweep_combine(x, parts, flags=flags)
    torch.cuda.synchronize()
    assert torch.equal(y, y_ref)
    ctx.close()


@pytest.mark.parametrize("variant", ["std", "lm", "rlm"])
@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_repeated_shard_applications_stay_bitwise(variant, mode):
    """A power iteration x <- K x / |K x| (as a Krylov solver applies the operator), each application swept in three
    chunks by three contexts of the problem and combined by a fourth, stays bitwise equal to lmdg_sweep."""
    import torch
    flags = _flags()[mode]
    p = random_problem(30, 8, 1.0, 7, ny=33)
    ref = _ctx(p, variant)
    shards = [_ctx(p, variant) for _ in range(3)]
    comb = _ctx(p, variant)
    sets, chunk, nbytes = ref.shard_layout(3, flags)
    parts = torch.empty(3 * nbytes, dtype=torch.uint8, device="cuda")
    x = torch.from_numpy(np.random.default_rng(5).standard_normal((p.nx, 4))).cuda()
    for it in range(25):
        y_ref = ref.sweep(x, flags=flags)
        for r, c in enumerate(shards):
            c.sweep_shard(x, parts, r, 3, flags)
        y = comb.sweep_combine(x, parts, flags=flags)
        torch.cuda.synchronize()
        assert torch.equal(y, y_ref), it
        x = y / torch.linalg.norm(y)
    for c in shards + [ref, comb]:
        c.close()


def test_sharded_sweep_on_one_rank():
    """The torch.distributed path of paper_1907_01027_gb300.shard.sharded_sweep on a process group of one rank (this
    test runs on one GPU): one chunk, the combine, lmdg_sweep's bits."""
    import os
    import socket
    import torch
    import torch.distributed as dist
    from paper_1907_01027_gb300 import SWEEP_SOURCE
    from paper_1907_01027_gb300.shard import sharded_sweep
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    store = dist.TCPStore("127.0.0.1", port, 1, True)
    dist.init_process_group("gloo", store=store, rank=0, world_size=1)
    try:
        p = random_problem(37, 8, 0.7, 4, ny=45)
        ctx = _ctx(p, "rlm")
        x = torch.from_numpy(np.random.default_rng(2).standard_normal((p.nx, 4))).cuda()
        for flags in (0, SWEEP_SOURCE):
            assert torch.equal(sharded_sweep(ctx, x, flags=flags), ctx.sweep(x, flags=flags))
        ctx.close()
    finally:
        dist.destroy_process_group()
