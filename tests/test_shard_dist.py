"""Angle sharding on CPU ranks (gloo): the split of the partial sets into chunks, the in-place all-gather of the
chunks, and a sharded operator application with the oracle producing each rank's partial sets.

The partial sets here are the library's: one per (quadrant, direction group), each the sum over its directions of
their contributions to the angular reduction (Q1-DG: w_l L_l^-1 M_l Phi; LMDG: w_l Psi0_l and the rows
Sigma L10 of Psi0_l, eq-nonrec-block), summed in set order after the exchange.  Every rank must end with the
single process's bits, and that result must be the oracle's operator.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1907_01027_gb300.shard import all_gather_chunks, chunk_range


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _spawn(fn, ws, *args):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=fn, args=(r, ws, port, q, *args)) for r in range(ws)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in range(ws)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return out


def _init(rank, ws, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)


@pytest.mark.parametrize("sets", [1, 4, 5, 20, 23])
@pytest.mark.parametrize("nshards", [1, 2, 3, 7, 30])
def test_chunk_range_partitions_the_sets(sets, nshards):
    seen = []
    for r in range(nshards):
        first, count = chunk_range(sets, nshards, r)
        assert count >= 0
        assert count <= -(-sets // nshards)
        seen += list(range(first, first + count))
    assert seen == list(range(sets))   # contiguous chunks in shard order, every set exactly once


def _gather_worker(rank, ws, port, q, chunk):
    _init(rank, ws, port)
    got = []
    for dtype in (torch.uint8, torch.float64):   # raw bytes (as the library's buffers travel) and values
        buf = torch.full((ws * chunk + 3,), 255, dtype=dtype)   # 3 elements past the chunks stay untouched
        buf[rank * chunk:(rank + 1) * chunk] = torch.arange(chunk, dtype=dtype) + 10 * rank
        all_gather_chunks(buf, chunk, rank, ws)
        got.append([int(v) for v in buf.tolist()])
    q.put((rank, got))
    dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
def test_all_gather_chunks_in_place(ws):
    chunk = 7
    want = [10 * r + k for r in range(ws) for k in range(chunk)] + [255] * 3
    for rank, got in _spawn(_gather_worker, ws, chunk):
        assert got == [want, want], rank


# ------------------------------------------------------------------ sharded operator application (oracle)
def _problem():
    from tests.helpers import random_problem
    return random_problem(6, 4, 0.5, 11, alpha=False, q_per_angle=False, ny=5)


def _sets(p, groups):
    """Direction lists of the partial sets: quadrant (+,+), (-,+), (-,-), (+,-) times ``groups`` groups."""
    quads = [[], [], [], []]
    for l in range(p.nang):
        ox, oy = p.ox[l], p.oy[l]
        quads[(0 if ox > 0 else 1) if oy > 0 else (2 if ox < 0 else 3)].append(l)
    out = []
    for dirs in quads:
        size = -(-len(dirs) // groups)
        out += [dirs[g * size:(g + 1) * size] for g in range(groups)]
    return out


def _partial(so, variant, dirs, X):
    """One partial set: the reduction's contributions of the directions ``dirs``, summed in their order."""
    acc = np.zeros((so.nx, 4))
    for l in dirs:
        if variant == "std":
            acc += so.p.w[l] * so.Linv(l, so.M(l, X))
        else:
            psi0 = so.L00inv(l, so.M0(l, X[:, 0]) + so.L01SigT(l, X[:, 1:]))
            acc[:, 0] += so.p.w[l] * psi0
            acc[:, 1:] += so.L(l, so._const(psi0))[:, 1:]
    return acc


def _combine(so, variant, X, parts, nsets):
    red = np.zeros((so.nx, 4))
    for s in range(nsets):          # fixed set order, whatever rank produced the set
        red += parts[s]
    if variant == "std":
        return X - red
    out = np.zeros((so.nx, 4))
    out[:, 0] = X[:, 0] - red[:, 0]
    out[:, 1:] = so.B11fast(X[:, 1:]) - red[:, 1:]
    return out


def _sharded_apply_worker(rank, ws, port, q, variant, groups):
    _init(rank, ws, port)
    from oracle.sweeps import SweepOracle
    p = _problem()
    so = SweepOracle(p, threads=1)
    X = np.random.default_rng(5).standard_normal((p.nx, 4))
    sets = _sets(p, groups)
    nsets = len(sets)
    chunk = -(-nsets // ws)
    buf = torch.zeros(ws * chunk * p.nx * 4, dtype=torch.float64)
    view = buf.view(ws * chunk, p.nx, 4).numpy()
    first, count = chunk_range(nsets, ws, rank)
    for s in range(first, first + count):
        view[s] = _partial(so, variant, sets[s], X)
    all_gather_chunks(buf, chunk * p.nx * 4, rank, ws)
    y = _combine(so, variant, X, view, nsets)
    q.put((rank, y))
    dist.destroy_process_group()


@pytest.mark.parametrize("variant", ["std", "lm"])
@pytest.mark.parametrize("ws,groups", [(2, 1), (2, 3), (3, 2)])
def test_sharded_apply_is_bitwise_the_single_process_one(variant, ws, groups):
    from oracle.sweeps import SweepOracle
    p = _problem()
    so = SweepOracle(p, threads=1)
    X = np.random.default_rng(5).standard_normal((p.nx, 4))
    sets = _sets(p, groups)
    single = _combine(so, variant, X, [_partial(so, variant, d, X) for d in sets], len(sets))
    ref = so.K(variant, X)
    assert np.abs(single - ref).max() <= 1e-13 * np.abs(ref).max()
    for rank, y in _spawn(_sharded_apply_worker, ws, variant, groups):
        assert np.array_equal(y, single), rank


# ------------------------------------------------------------------ shard.sharded_sweep on gloo ranks
class _OracleShardContext:
    """Stands in for a Context in shard.sharded_sweep on the CPU: the same three calls (layout, one chunk's partial
    sets into a byte buffer, the combine), their arithmetic done by the oracle (test infrastructure only)."""

    def __init__(self, variant, groups):
        from oracle.sweeps import SweepOracle
        self.p = _problem()
        self.so = SweepOracle(self.p, threads=1)
        self.variant = variant
        self.sets = _sets(self.p, groups)

    def shard_layout(self, nshards, flags=0):
        chunk = -(-len(self.sets) // nshards)
        return len(self.sets), chunk, chunk * self.p.nx * 4 * 8

    def sweep_shard(self, x, parts, shard, nshards, flags=0):
        _, chunk, _ = self.shard_layout(nshards)
        view = parts.view(torch.float64).view(nshards * chunk, self.p.nx, 4).numpy()
        first, count = chunk_range(len(self.sets), nshards, shard)
        X = x.numpy()
        for s in range(first, first + count):
            view[s] = _partial(self.so, self.variant, self.sets[s], X)

    def sweep_combine(self, x, parts, y=None, flags=0):
        view = parts.view(torch.float64).view(-1, self.p.nx, 4).numpy()
        return torch.from_numpy(_combine(self.so, self.variant, x.numpy(), view, len(self.sets)))


def _sharded_sweep_worker(rank, ws, port, q, variant, groups):
    _init(rank, ws, port)
    from paper_1907_01027_gb300.shard import sharded_sweep
    ctx = _OracleShardContext(variant, groups)
    x = torch.from_numpy(np.random.default_rng(5).standard_normal((ctx.p.nx, 4)))
    q.put((rank, sharded_sweep(ctx, x).numpy()))
    dist.destroy_process_group()


@pytest.mark.parametrize("variant", ["std", "lm"])
@pytest.mark.parametrize("ws,groups", [(2, 2), (3, 1)])
def test_sharded_sweep_helper_on_gloo_ranks(variant, ws, groups):
    """paper_1907_01027_gb300.shard.sharded_sweep itself (layout, this rank's chunk, in-place all-gather, combine)
    across ranks: every rank gets the single process's bits."""
    ctx = _OracleShardContext(variant, groups)
    X = np.random.default_rng(5).standard_normal((ctx.p.nx, 4))
    single = _combine(ctx.so, variant, X, [_partial(ctx.so, variant, d, X) for d in ctx.sets], len(ctx.sets))
    for rank, y in _spawn(_sharded_sweep_worker, ws, variant, groups):
        assert np.array_equal(y, single), rank
