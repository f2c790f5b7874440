"""Angle sharding over torch.distributed ranks, one GPU per rank.

The sweep is independent per direction (Section 2.1.1: L is block diagonal over the directions) and only the
angular reduction couples the directions.  The library forms a sweep's reduction from partial sets, one per
(quadrant, direction group) of its launch shape, and sums them in a fixed order in the epilogue.  Sharding splits
the sets into one contiguous chunk per rank (``lmdg_shard_layout``): each rank sweeps the whole mesh for the
directions of its chunk, the ranks all-gather the chunks in place, and every rank runs the same epilogue, so the
result is bitwise the one GPU's.  The stored angular unknowns of a storing sweep are sharded by direction.

Only argument marshalling and the collective live here; every sweep and epilogue runs in the library's kernels.
"""


def chunk_range(sets, nshards, shard):
    """(first set, number of sets) of chunk ``shard``: chunks of ceil(sets / nshards) sets, the last ones shorter
    or empty -- the split the library applies (``lmdg_shard_layout``)."""
    chunk = -(-sets // nshards)
    first = min(sets, shard * chunk)
    return first, min(sets, (shard + 1) * chunk) - first


def all_gather_chunks(buf, chunk_numel, rank, world, group=None):
    """In-place all-gather of a flat tensor holding ``world`` chunks of ``chunk_numel`` elements: on entry chunk
    ``rank`` holds this rank's data, on return every chunk holds its owner's (any backend that implements
    all_gather_into_tensor; gloo on the CPU, NCCL on the GPU, where it is ordered on the current stream)."""
    import torch.distributed as dist
    mine = buf[rank * chunk_numel:(rank + 1) * chunk_numel].clone()
    dist.all_gather_into_tensor(buf[:world * chunk_numel], mine, group=group)


def sharded_sweep(ctx, x, y=None, flags=0, group=None):
    """One application of the reduced operator -- lmdg_sweep's y = K x, or K x - b with SWEEP_SOURCE -- with the
    directions split across the ranks of ``group`` (default: the world), one GPU per rank: this rank sweeps its
    chunk of the partial sets (``lmdg_sweep_shard``), the chunks are all-gathered in place, and the epilogue
    (``lmdg_sweep_combine``) gives every rank the bits one GPU's ``lmdg_sweep`` gives.  ``ctx`` is this rank's
    :class:`~paper_1907_01027_gb300.lmdg.Context` of the problem (set up with the same arguments on every rank);
    ``x`` a CUDA tensor [N][4] of float64, the same on every rank."""
    import torch
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    _, _, nbytes = ctx.shard_layout(world, flags)
    parts = torch.empty(world * nbytes, dtype=torch.uint8, device=x.device)
    ctx.sweep_shard(x, parts, rank, world, flags)
    if world > 1:
        all_gather_chunks(parts, nbytes, rank, world, group)
    return ctx.sweep_combine(x, parts, y, flags)


__all__ = ["chunk_range", "all_gather_chunks", "sharded_sweep"]
