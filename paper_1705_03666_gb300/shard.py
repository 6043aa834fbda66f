"""Sharding of stage one across ranks, and its one exchange step.

Interface nodes are independent units, and within a node any range of path
indices is reproducible anywhere (counter-based streams), so stage one shards
without communication: by node (block distribution) or by path range.  The
only exchange before stage two is an all-gather of per-node (count, mean, M2)
triples, merged with Chan's formula where one node's paths span ranks.
Works with any torch.distributed backend (gloo on CPU tensors, NCCL on CUDA
tensors); the solves themselves run in libpdd.so.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def node_block(n: int, world: int, rank: int) -> tuple[int, int]:
    """Half-open node range of `rank` in a block distribution of n nodes."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def path_block(n_paths: int, world: int, rank: int) -> tuple[int, int]:
    """Half-open path-index range of `rank` (same rule as node_block)."""
    return node_block(n_paths, world, rank)


def triples(mean: torch.Tensor, se: torch.Tensor, count: torch.Tensor) -> torch.Tensor:
    """(count, mean, M2) per node from mean, standard error and count
    (M2 = se^2 * count * (count - 1))."""
    c = count.to(torch.float64)
    return torch.stack([c, mean.to(torch.float64), se.to(torch.float64) ** 2 * c * (c - 1)], 1)


def chan_merge(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """Merge two [n, 3] (count, mean, M2) tables (Chan, Golub, LeVeque)."""
    na, ma, m2a = a.unbind(1)
    nb, mb, m2b = b.unbind(1)
    nt = na + nb
    safe = torch.where(nt > 0, nt, torch.ones_like(nt))
    d = mb - ma
    mean = ma + d * nb / safe
    m2 = m2a + m2b + d * d * na * nb / safe
    return torch.stack([nt, mean, m2], 1)


def finalize(t: torch.Tensor):
    """mean, standard error, count from a (count, mean, M2) table."""
    c, m, m2 = t.unbind(1)
    se = torch.where(c > 1, torch.sqrt(m2 / (c - 1).clamp(min=1) / c.clamp(min=1)),
                     torch.zeros_like(m))
    return m, se, c.to(torch.int64)


def allgather_nodes(local: torch.Tensor, n_total: int, group=None) -> torch.Tensor:
    """Node sharding: every rank holds the [n_local, 3] triples of its node
    block; returns the full [n_total, 3] table on every rank."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    lo, hi = node_block(n_total, world, rank)
    assert local.shape[0] == hi - lo
    width = max(node_block(n_total, world, r)[1] - node_block(n_total, world, r)[0]
                for r in range(world))
    pad = torch.zeros((width, 3), dtype=torch.float64, device=local.device)
    pad[:hi - lo] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    out = []
    for r, p in enumerate(parts):
        a, b = node_block(n_total, world, r)
        out.append(p[:b - a])
    return torch.cat(out)


def allreduce_paths(local: torch.Tensor, group=None) -> torch.Tensor:
    """Path-range sharding: every rank holds triples of all nodes over its own
    path range; returns the merged table (ranks merged in rank order, so the
    result does not depend on arrival order)."""
    world = dist.get_world_size(group)
    parts = [torch.empty_like(local) for _ in range(world)]
    dist.all_gather(parts, local.contiguous(), group=group)
    acc = parts[0]
    for p in parts[1:]:
        acc = chan_merge(acc, p)
    return acc
