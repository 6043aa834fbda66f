"""Multi-rank stage one on CPU (gloo, world size 2): node sharding and
path-range sharding with the one exchange step (all-gather of per-node
(count, mean, M2) triples, Chan merge) reproduce the single-process estimate.
The per-rank solves use the FP64 oracle (no GPU here)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1705_03666_gb300 import shard, workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, mode, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    w = W.workload(2)
    nodes = w["nodes"][::256]
    n = len(nodes)
    kw = dict(seed=w["seed"], dt=1e-3, n_threads=1)
    if mode == "nodes":
        lo, hi = shard.node_block(n, world, rank)
        r = oracle.interface_solve(w["prob"], nodes[lo:hi], node_ids=np.arange(lo, hi),
                                   n_paths=600, **kw)
        t = shard.triples(torch.from_numpy(r["mean"]), torch.from_numpy(r["se"]),
                          torch.from_numpy(r["n"]))
        full = shard.allgather_nodes(t, n)
    elif mode == "copies":
        # the benchmark's multi-GPU layout: rank r solves copy r of the node
        # list (node ids r n .. r n + n - 1), the all-gather assembles all
        off, total = shard.copy_block(n, world, rank)
        r = oracle.interface_solve(w["prob"], nodes, node_ids=np.arange(off, off + n),
                                   n_paths=600, **kw)
        t = shard.triples(torch.from_numpy(r["mean"]), torch.from_numpy(r["se"]),
                          torch.from_numpy(r["n"]))
        full = shard.allgather_nodes(t, total)
    else:
        lo, hi = shard.path_block(600, world, rank)
        r = oracle.interface_solve(w["prob"], nodes, n_paths=hi - lo, path_offset=lo, **kw)
        t = shard.triples(torch.from_numpy(r["mean"]), torch.from_numpy(r["se"]),
                          torch.from_numpy(r["n"]))
        full = shard.allreduce_paths(t)
    m, se, c = shard.finalize(full)
    np.save(os.path.join(out_dir, f"{mode}_{rank}.npy"), torch.stack([m, se, c.double()]).numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["nodes", "paths", "copies"])
def test_two_rank_stage_one_matches_single_process(tmp_path, mode):
    import oracle
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), mode, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    w = W.workload(2)
    nodes = w["nodes"][::256]
    if mode == "copies":
        nodes = np.concatenate([nodes] * world)
    ref = oracle.interface_solve(w["prob"], nodes, seed=w["seed"], dt=1e-3, n_paths=600)
    for r in range(world):
        got = np.load(tmp_path / f"{mode}_{r}.npy")
        np.testing.assert_allclose(got[0], ref["mean"], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(got[1], ref["se"], rtol=1e-9)
        assert np.array_equal(got[2], ref["n"].astype(np.float64))


def test_blocks_cover_exactly():
    for n in (0, 1, 7, 4096):
        for world in (1, 2, 3, 8):
            ranges = [shard.node_block(n, world, r) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
