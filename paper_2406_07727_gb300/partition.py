"""Vertex-partitioned three-hop search over several GPUs, one process per GPU.

The paths of a query are split by their hop-1 vertex: rank r of W searches
only the paths s -> u -> v -> t with u % W == r (mhr_query_opts.part_count /
part_index), so every path belongs to exactly one rank.  The ranks' K-best
lists (K x 24 bytes per query) are all-gathered and merged by the library's
GPU tree merge (mhr_merge_paths, Alg. 2), and every rank ends with the
unpartitioned result.  Each rank holds the whole graph: what is split is the
middle-join work, one part per GPU.

This module only drives: the search and the merge run in the library's
kernels; torch.distributed moves the lists (NCCL between GPUs).
"""

from __future__ import annotations

from . import _mhr


def part_options(opts, world: int, rank: int) -> dict:
    """The query options of rank `rank` of `world`: its part of the paths."""
    o = dict(opts or {})
    if world > 1:
        o["part_count"] = int(world)
        o["part_index"] = int(rank)
    return o


def gather_parts(out, n_out, group=None):
    """All-gather every rank's lists: (out [nq, K*24] uint8, n_out [nq] int32)
    -> (parts [W, nq, K*24], counts [W, nq]) in rank order."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    outs = [torch.empty_like(out) for _ in range(world)]
    cnts = [torch.empty_like(n_out) for _ in range(world)]
    dist.all_gather(outs, out.contiguous(), group=group)
    dist.all_gather(cnts, n_out.contiguous(), group=group)
    return torch.stack(outs), torch.stack(cnts)


def topk_paths_partitioned(G, S, T, K: int, opts=None, group=None, stream=None):
    """Exact three-hop top K of the queries (S, T: device tensors) with the
    paths partitioned over the process group's ranks; every rank returns the
    full result (device tensors out [nq, K*24] uint8, n_out [nq] int32)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return _mhr.mhr_topk_paths_batched(G, S, T, K, opts=opts, stream=stream)
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    out, n_out = _mhr.mhr_topk_paths_batched(G, S, T, K, opts=part_options(opts, world, rank), stream=stream)
    if world == 1:
        return out, n_out
    parts, counts = gather_parts(out, n_out, group)
    return _mhr.mhr_merge_paths(parts, counts, K, stream=stream)
