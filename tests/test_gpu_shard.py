"""Angle sharding through the C ABI on one GPU.

(1) Sweeping every chunk of the partial sets with lmdg_sweep_shard and combining them with lmdg_sweep_combine gives
lmdg_sweep's result bit for bit, for every scheme and arithmetic, with chunks that hold several sets, one set or
none.  (2) A context sharded with lmdg_set_shard solves bit for bit like an unsharded one; here the exchange
callback, instead of all-gathering from other GPUs, sweeps the other chunks itself through contexts of the same
problem (what the other ranks would have computed), so the multi-GPU solve path runs on one GPU.
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
    assert chunk == -(-sets // nshards) and nbytes % 16 == 0
    parts = torch.empty(nshards * nbytes, dtype=torch.uint8, device="cuda")
    for r in reversed(range(nshards)):   # any order: each chunk is written by its own shard only
        ctx.sweep_shard(x, parts, r, nshards, flags)
    y = ctx.sweep_combine(x, parts, flags=flags)
    torch.cuda.synchronize()
    assert torch.equal(y, y_ref)
    ctx.close()


def _emulated(p, variant, nshards, **kw):
    """Context 0 sharded over nshards, its exchange sweeping chunks 1.. through contexts of its own."""
    ctxs = [_ctx(p, variant, **kw) for _ in range(nshards)]
    lib = ctxs[0].lib
    calls = []

    def exchange(parts, chunk_bytes, n, x, flags, stream):
        calls.append(flags)
        for r in range(1, n):
            if lib.lmdg_sweep_shard(ctxs[r].h, x, parts, r, n, flags, stream):
                return 1
        return 0

    ctxs[0].set_shard(0, nshards, exchange)
    return ctxs, calls


@pytest.mark.parametrize("variant", ["std", "lm", "rlm"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sharded_solve_is_bitwise_the_unsharded_solve(variant, prec):
    from paper_1907_01027_gb300 import FP32, FP64, RESID_F32X2
    kw = dict(precision=FP64, tol=1e-11) if prec == "fp64" else dict(precision=FP32, resid=RESID_F32X2, tol=1e-9)
    p = random_problem(30, 8, 1.0, 7, ny=33)
    ref = _ctx(p, variant, **kw)
    x1, phi1, st1, rc1 = ref.solve()
    ctxs, calls = _emulated(p, variant, 3, **kw)
    x0, phi0, st0, rc0 = ctxs[0].solve()
    assert rc0 == rc1 == 0
    assert st0["iters"] == st1["iters"] and len(calls) == st0["sweeps_fp64"] + st0["sweeps_fp32"] + st0["sweeps_f32x2"]
    assert np.array_equal(x0, x1) and np.array_equal(phi0, phi1)
    # the sharded context sweeps a third of the partial sets: undoing the sharding restores the full sweep
    ctxs[0].set_shard(0, 1)
    x2, phi2, _, _ = ctxs[0].solve()
    assert np.array_equal(x2, x1) and np.array_equal(phi2, phi1)
    for c in ctxs + [ref]:
        c.close()


def test_sharded_context_refuses_the_adjoint_and_reports_a_failed_exchange():
    from paper_1907_01027_gb300 import LmdgError
    from paper_1907_01027_gb300.lmdg import ERR_EXCHANGE, ERR_STATE
    p = random_problem(12, 4, 1.0, 9, alpha=False, q_per_angle=False)
    ctxs, _ = _emulated(p, "std", 2)
    with pytest.raises(LmdgError) as e:
        ctxs[0].adjoint(np.ones(p.nx))
    assert e.value.code == ERR_STATE
    ctxs[0].set_shard(0, 2, lambda *a: 1)
    with pytest.raises(LmdgError) as e:
        ctxs[0].sweep(np.ones((p.nx, 4)))
    assert e.value.code == ERR_EXCHANGE
    ctxs[0].set_shard(0, 1)
    ctxs[0].sweep(np.ones((p.nx, 4)))   # the context stays usable
    for c in ctxs:
        c.close()
