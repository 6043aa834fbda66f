"""Checkpoint and resume of an interface solve.

Per node, the running (count, mean, M2) triple and the index of the next path
form a complete checkpoint.  Path p of node j draws its random numbers from
the counter (p, j) under the seed and nothing else, so a later call with
path_offset = next path continues the same sample, on any device or rank,
and merging the triples (Chan, Golub and LeVeque) gives the estimate that one
longer run would give, up to rounding.  A checkpoint records a digest of
everything that fixes the paths (problem, nodes, seed, dt, precision, bridge,
step cap); resuming with different settings is an error.

Host logic only: the solves are the caller's (`Context.interface_solve`).
"""
from __future__ import annotations

import hashlib
import os
import zipfile

import numpy as np
import torch

from . import shard


def _np(x) -> np.ndarray:
    if isinstance(x, torch.Tensor):
        return x.detach().cpu().numpy()
    return np.asarray(x)


def run_digest(prob: dict, nodes, *, seed: int, dt: float, precision: str = "fp32",
               bridge: bool = True, max_steps: int = 2**31 - 1) -> str:
    """Digest of the settings that fix every path of a run."""
    h = hashlib.sha1()
    for k in sorted(prob):
        v = prob[k]
        h.update(k.encode())
        if isinstance(v, (list, tuple, np.ndarray)):
            h.update(np.ascontiguousarray(np.asarray(v, dtype=np.float64)).tobytes())
        else:
            h.update(repr(v).encode())
    h.update(np.ascontiguousarray(_np(nodes), dtype=np.float64).tobytes())
    h.update(repr((int(seed) & (2**64 - 1), float(dt), str(precision), bool(bridge),
                   int(max_steps))).encode())
    return h.hexdigest()


class Checkpoint:
    """Running per-node (count, mean, M2) table and the next path index."""

    def __init__(self, digest: str, n_nodes: int, next_path: int = 0, table=None):
        self.digest = digest
        self.next_path = int(next_path)
        self.table = (torch.zeros((n_nodes, 3), dtype=torch.float64) if table is None
                      else torch.as_tensor(np.asarray(table, dtype=np.float64)).clone())
        if self.table.shape != (n_nodes, 3):
            raise ValueError(f"table shape {tuple(self.table.shape)} for {n_nodes} nodes")

    @classmethod
    def start(cls, prob: dict, nodes, **run) -> "Checkpoint":
        return cls(run_digest(prob, nodes, **run), len(_np(nodes)))

    def add(self, res: dict, n_paths: int) -> None:
        """Merge the result of a solve over paths [next_path, next_path +
        n_paths) (mean, se, n per node) and advance next_path."""
        t = shard.triples(torch.from_numpy(_np(res["mean"]).astype(np.float64)),
                          torch.from_numpy(_np(res["se"]).astype(np.float64)),
                          torch.from_numpy(_np(res["n"]).astype(np.int64)))
        if t.shape != self.table.shape:
            raise ValueError(f"result has {t.shape[0]} nodes, checkpoint {self.table.shape[0]}")
        self.table = shard.chan_merge(self.table, t)
        self.next_path += int(n_paths)

    def result(self) -> dict:
        m, se, c = shard.finalize(self.table)
        return {"mean": m.numpy(), "se": se.numpy(), "n": c.numpy(),
                "next_path": self.next_path}

    def save(self, path: str) -> None:
        """Write atomically and durably: a temporary file, flushed to the disk,
        renamed over `path`, and the directory entry flushed too, so that a
        crash leaves either the previous checkpoint or this one."""
        tmp = f"{path}.tmp"
        with open(tmp, "wb") as f:
            np.savez(f, table=self.table.numpy(), next_path=np.int64(self.next_path),
                     digest=np.array(self.digest))
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, path)
        d = os.open(os.path.dirname(os.path.abspath(path)), os.O_RDONLY)
        try:
            os.fsync(d)
        finally:
            os.close(d)

    @classmethod
    def load(cls, path: str) -> "Checkpoint":
        try:
            with np.load(path) as z:
                table = z["table"]
                ck = cls(str(z["digest"]), table.shape[0], int(z["next_path"]), table)
        except (OSError, ValueError, KeyError, EOFError, zipfile.BadZipFile) as e:  # truncated
            raise ValueError(f"checkpoint file {path} is unreadable (truncated or corrupt): "
                             f"{e}") from e
        if table.ndim != 2 or table.shape[1] != 3:
            raise ValueError(f"checkpoint file {path} holds a table of shape {table.shape}")
        return ck

    def check(self, prob: dict, nodes, **run) -> None:
        if run_digest(prob, nodes, **run) != self.digest:
            raise ValueError("checkpoint was written for another problem, node set or "
                             "run settings")


def solve_resumable(solve, prob: dict, nodes, *, seed: int, dt: float, n_paths: int,
                    piece: int, path: str | None = None, precision: str = "fp32",
                    bridge: bool = True, max_steps: int = 2**31 - 1) -> dict:
    """n_paths paths per node in pieces of at most `piece` paths, through
    `solve(nodes, seed=, dt=, n_paths=, path_offset=, precision=, bridge=,
    max_steps=)` (e.g. a Context's interface_solve), writing the checkpoint to
    `path` after each piece; if `path` exists the run continues from it.
    Returns the merged mean, se, n and next_path."""
    run = dict(seed=seed, dt=dt, precision=precision, bridge=bridge, max_steps=max_steps)
    if piece < 1:
        raise ValueError("piece must be >= 1")
    if path is not None and os.path.exists(path):
        ck = Checkpoint.load(path)
        ck.check(prob, nodes, **run)
    else:
        ck = Checkpoint.start(prob, nodes, **run)
    if ck.next_path > n_paths:
        raise ValueError(f"checkpoint already holds {ck.next_path} paths per node")
    while ck.next_path < n_paths:
        k = min(piece, n_paths - ck.next_path)
        res = solve(nodes, n_paths=k, path_offset=ck.next_path, **run)
        ck.add(res, k)
        if path is not None:
            ck.save(path)
    return ck.result()
