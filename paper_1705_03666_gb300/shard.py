"""Sharding of stage one across ranks, and its one exchange step.

Interface nodes are independent units, and within a node any range of path
indices is reproducible anywhere (counter-based streams), so stage one shards
without communication: by node (block distribution) or by path range.  The
only exchange before stage two is an all-gather of per-node (count, mean, M2)
triples, merged with Chan's formula where one node's paths span ranks.
Works with any torch.distributed backend (gloo on CPU tensors, NCCL on CUDA
tensors); the solves themselves run in libpdd.so.  The same exchange can go
through a key-value store with a deadline instead (publish / collect), so
that the survivors of a lost rank carry on without it.
"""
from __future__ import annotations

import time

import numpy as np
import torch
import torch.distributed as dist


def node_block(n: int, world: int, rank: int) -> tuple[int, int]:
    """Half-open node range of `rank` in a block distribution of n nodes."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def copy_block(n: int, world: int, rank: int) -> tuple[int, int]:
    """Weak scaling by node blocks: the run's node list is `world` copies of
    an n-node list, copy r being nodes [r n, (r + 1) n) with their own
    stream indices; `rank` solves its copy (node_offset = r n) and the
    all-gather assembles the world x n table.  Returns (node_offset, total)."""
    return rank * n, world * n


def path_block(n_paths: int, world: int, rank: int) -> tuple[int, int]:
    """Half-open path-index range of `rank` (same rule as node_block)."""
    return node_block(n_paths, world, rank)


def triples(mean: torch.Tensor, se: torch.Tensor, count: torch.Tensor) -> torch.Tensor:
    """(count, mean, M2) per node from mean, standard error and count
    (M2 = se^2 * count * (count - 1))."""
    c = count.to(torch.float64)
    return torch.stack([c, mean.to(torch.float64), se.to(torch.float64) ** 2 * c * (c - 1)], 1)


def chan_merge(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """Merge two [n, 3] (count, mean, M2) tables (Chan, Golub, LeVeque).  A
    row with count 0 on one side takes the other side's row as it is, so an
    empty side's mean (NaN where nothing was sampled) never enters the
    arithmetic."""
    na, ma, m2a = a.unbind(1)
    nb, mb, m2b = b.unbind(1)
    nt = na + nb
    safe = torch.where(nt > 0, nt, torch.ones_like(nt))
    d = mb - ma
    mean = ma + d * nb / safe
    m2 = m2a + m2b + d * d * na * nb / safe
    merged = torch.stack([nt, mean, m2], 1)
    merged = torch.where((na == 0)[:, None], b, merged)
    return torch.where((nb == 0)[:, None], a, merged)


def finalize(t: torch.Tensor):
    """mean, standard error, count from a (count, mean, M2) table; a row
    with count 0 (no sample: a node nobody supplied) gives NaN mean and se,
    as the library's own finalisation does."""
    c, m, m2 = t.unbind(1)
    nan = torch.full_like(m, float("nan"))
    se = torch.where(c > 1, torch.sqrt(m2 / (c - 1).clamp(min=1) / c.clamp(min=1)),
                     torch.zeros_like(m))
    return torch.where(c > 0, m, nan), torch.where(c > 0, se, nan), c.to(torch.int64)


def allgather_nodes(local: torch.Tensor, n_total: int, group=None) -> torch.Tensor:
    """Node sharding: every rank holds the [n_local, 3] triples of its node
    block; returns the full [n_total, 3] table on every rank."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    lo, hi = node_block(n_total, world, rank)
    if local.shape[0] != hi - lo:
        raise ValueError(f"rank {rank} holds {local.shape[0]} rows for block [{lo}, {hi})")
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


# ---------------------------------------------------------------------------
# Exchange through a key-value store with a deadline, for runs that must
# survive the loss of a rank.  A rank that fails between steps only takes its
# own units with it (the paper's remark on fault tolerance in Sec. 2): with
# path-range sharding the survivors' samples still give an unbiased estimate
# with a wider standard error; with node sharding the lost block is
# recomputed by the survivors, and because every path's random numbers come
# from (seed, node id, path index) the recomputed values are the ones the
# lost rank would have produced.  No collective is involved, so a missing
# rank cannot block the others beyond the deadline.
# ---------------------------------------------------------------------------

def publish(store, tag: str, rank: int, table: torch.Tensor) -> None:
    """Post this rank's [rows, 3] (count, mean, M2) table under `tag`."""
    t = table.detach().to("cpu", torch.float64).contiguous()
    store.set(f"{tag}/{rank}", t.numpy().tobytes())


def collect(store, tag: str, ranks, timeout_s: float, poll_s: float = 0.01):
    """Wait up to `timeout_s` seconds for the tables that `ranks` publish
    under `tag`.  Returns ({rank: [rows, 3] table} for the ranks that
    published, sorted list of the ranks that did not)."""
    deadline = time.monotonic() + timeout_s
    pending = sorted(set(int(r) for r in ranks))
    got = {}
    while True:
        for r in list(pending):
            key = f"{tag}/{r}"
            if store.check([key]):
                buf = np.frombuffer(store.get(key), dtype=np.float64).copy()
                got[r] = torch.from_numpy(buf).reshape(-1, 3)
                pending.remove(r)
        if not pending or time.monotonic() >= deadline:
            return got, pending
        time.sleep(poll_s)


def agree(store, tag: str, got: dict, lost) -> tuple[dict, list, list]:
    """Make every rank act on the same (alive, lost) split after `collect`.

    Each rank's collect has its own deadline, so a rank that published close
    to it can be seen by one survivor and missed by another.  The first rank
    to get here writes its own view under `tag`/view (compare-and-set on an
    unset key, so only one write succeeds) and every rank adopts the stored
    view.  Returns (the agreed alive ranks' tables, agreed lost ranks,
    agreed alive ranks); a table this rank's own collect missed is read from
    the store (the writer saw it published).  A rank absent from the agreed
    alive list has been declared lost: its table is not used and it
    recomputes nothing."""
    alive = sorted(int(r) for r in got)
    mine = ",".join(str(r) for r in alive) + "|" + ",".join(str(int(r)) for r in sorted(lost))
    stored = store.compare_set(f"{tag}/view", "", mine)
    view = stored.decode() if isinstance(stored, (bytes, bytearray)) else str(stored)
    a, l = view.split("|")
    alive_a = [int(r) for r in a.split(",") if r]
    lost_a = [int(r) for r in l.split(",") if r]
    out = {}
    for r in alive_a:
        if r in got:
            out[r] = got[r]
        else:
            buf = np.frombuffer(store.get(f"{tag}/{r}"), dtype=np.float64).copy()
            out[r] = torch.from_numpy(buf).reshape(-1, 3)
    return out, lost_a, alive_a


def merge_surviving_paths(got: dict) -> torch.Tensor:
    """Path-range sharding after `collect`: merge the surviving ranks' tables
    in rank order (the result is the estimate over their path ranges)."""
    if not got:
        raise RuntimeError("no rank published its table")
    ranks = sorted(got)
    acc = got[ranks[0]]
    for r in ranks[1:]:
        acc = chan_merge(acc, got[r])
    return acc


def lost_node_share(n_total: int, world: int, lost, alive, rank: int) -> list[tuple[int, int]]:
    """Node sharding: the half-open node ranges `rank` (a survivor) recomputes
    when the ranks in `lost` are gone.  Each lost rank's block is split over
    the survivors in rank order by the block rule."""
    alive = sorted(alive)
    me = alive.index(rank)
    out = []
    for r in sorted(lost):
        lo, hi = node_block(n_total, world, r)
        a, b = node_block(hi - lo, len(alive), me)
        if b > a:
            out.append((lo + a, lo + b))
    return out


def assemble_nodes(n_total: int, world: int, got: dict, lost=(), redo: dict | None = None):
    """Node sharding: the full [n_total, 3] table from the blocks that
    arrived (`got`, keyed by owning rank) and, for the `lost` ranks' blocks,
    the survivors' recomputed rows (`redo`, keyed by survivor: its
    `lost_node_share` pieces, concatenated in order).  Rows nobody supplied
    keep count 0 (finalize gives NaN mean and se, count 0 there)."""
    out = torch.zeros((n_total, 3), dtype=torch.float64)
    for r, t in got.items():
        lo, hi = node_block(n_total, world, r)
        if t.shape[0] != hi - lo:
            raise ValueError(f"rank {r} published {t.shape[0]} rows for block [{lo}, {hi})")
        out[lo:hi] = t
    alive = sorted(got)
    for r, t in (redo or {}).items():
        pieces = lost_node_share(n_total, world, lost, alive, r)
        if t.shape[0] != sum(b - a for a, b in pieces):
            raise ValueError(f"rank {r} recomputed {t.shape[0]} rows for pieces {pieces}")
        k = 0
        for a, b in pieces:
            out[a:b] = t[k:k + b - a]
            k += b - a
    return out
