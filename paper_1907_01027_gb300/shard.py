"""Angle sharding over torch.distributed ranks, one GPU per rank.

The sweep is independent per direction (Section 2.1.1: L is block diagonal over the directions) and only the
angular reduction couples the directions.  The library forms a sweep's reduction from partial sets, one per
(quadrant, direction group) of its launch shape, and sums them in a fixed order in the epilogue.  Sharding splits
the sets into one contiguous chunk per rank (``lmdg_shard_layout``): each rank sweeps the whole mesh for the
directions of its chunk, the ranks all-gather the chunks in place (the exchange callback of ``lmdg_set_shard``),
and every rank runs the same epilogue, so the result is bitwise the one GPU's.  GMRES vectors are replicated (every
rank runs the same iterations on the same data); the stored angular unknowns are sharded by direction.

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


class _DeviceBytes:
    """A device allocation of the library seen by torch as a uint8 tensor (no copy)."""

    def __init__(self, ptr, nbytes):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False), "version": 3}


def attach(ctx, group=None):
    """Shard ``ctx`` (a :class:`~paper_1907_01027_gb300.lmdg.Context` on this rank's GPU, set up with the same
    problem and options on every rank) over the ranks of ``group``: every later sweep of the context -- ``sweep``,
    ``solve`` and its recovery sweep -- sweeps this rank's chunk of the directions and all-gathers the partial sets
    before its epilogue.  Returns (rank, world)."""
    import torch
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    dev = torch.device("cuda", torch.cuda.current_device())

    def exchange(parts, chunk_bytes, nshards, x, flags, stream):
        try:
            buf = torch.as_tensor(_DeviceBytes(parts, nshards * chunk_bytes), device=dev)
            st = torch.cuda.ExternalStream(stream, device=dev) if stream else torch.cuda.default_stream(dev)
            with torch.cuda.stream(st):
                all_gather_chunks(buf, chunk_bytes, rank, nshards, group)
            return 0
        except Exception:   # reported to the caller of the sweep as LMDG_ERR_EXCHANGE
            return 1

    ctx.set_shard(rank, world, exchange if world > 1 else None)
    return rank, world


def detach(ctx):
    """Undo :func:`attach`: the context sweeps every direction again."""
    ctx.set_shard(0, 1)


__all__ = ["chunk_range", "all_gather_chunks", "attach", "detach"]
