"""Multi-GPU plumbing around the search (host side, torch.distributed).

Queries are independent (Algorithm 1 runs per query), so the natural multi-GPU
form is replicas: every rank holds the whole index and searches its own slice of
the queries; there is no exchange on the data path.  For an index larger than
one GPU the base is split into id ranges, every rank searches every query on its
shard, and one exchange merges the per-shard top-k lists by (dist, id).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [start, end) slice of n items for `rank` (sizes differ by at most one)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def merge_topk(ids: torch.Tensor, dists: torch.Tensor, k: int):
    """Per row, the k smallest (dist, id) among candidate lists concatenated along dim 1.
    Entries with id < 0 are empty.  Returns (ids [rows, k], dists [rows, k])."""
    big = torch.iinfo(torch.int64).max
    key_id = torch.where(ids < 0, torch.full_like(ids, -1), ids).to(torch.int64)
    d = torch.where(ids < 0, torch.full_like(dists, float("inf")), dists)
    tie = torch.where(key_id < 0, torch.full_like(key_id, big), key_id)
    o1 = torch.argsort(tie, dim=1, stable=True)
    d1 = torch.gather(d, 1, o1)
    i1 = torch.gather(key_id, 1, o1)
    o2 = torch.argsort(d1, dim=1, stable=True)
    d2 = torch.gather(d1, 1, o2)[:, :k]
    i2 = torch.gather(i1, 1, o2)[:, :k]
    return i2.to(torch.int32), d2


def gather_rows(t: torch.Tensor, n_total: int, group=None) -> torch.Tensor:
    """All-gather row slices produced under shard_range(n_total, rank, world), in rank order."""
    world = dist.get_world_size(group)
    rows = [shard_range(n_total, r, world) for r in range(world)]
    cap = max(e - s for s, e in rows)
    pad = torch.zeros((cap,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
    pad[: t.shape[0]] = t
    bufs = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(bufs, pad, group=group)
    return torch.cat([b[: e - s] for b, (s, e) in zip(bufs, rows)], 0)


def merge_shards(ids: torch.Tensor, dists: torch.Tensor, id_offset: int, k: int, group=None):
    """Base-sharded search: each rank holds its shard's top-k (local ids) for every
    query; one all-gather exchanges them and every rank returns the global top-k."""
    gids = torch.where(ids >= 0, ids.to(torch.int64) + id_offset, torch.full_like(ids, -1, dtype=torch.int64))
    world = dist.get_world_size(group)
    all_i = [torch.empty_like(gids) for _ in range(world)]
    all_d = [torch.empty_like(dists) for _ in range(world)]
    dist.all_gather(all_i, gids, group=group)
    dist.all_gather(all_d, dists, group=group)
    return merge_topk(torch.cat(all_i, 1), torch.cat(all_d, 1), k)
