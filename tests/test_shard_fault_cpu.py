"""Loss of a rank in sharded stage one, on CPU processes (no GPU, no
collective): ranks exchange their (count, mean, M2) tables through a TCP
key-value store with a deadline, and one rank fails on the host (raises)
after its solve and before it publishes.  The survivors notice the missing
table at the deadline and carry on (Sec. 2: the loss of a processor only
loses samples):
  * node sharding: they recompute the lost block between them, and the
    result equals the single-process estimate (counter-based streams);
  * path-range sharding: the estimate over the survivors' paths is the
    single-process estimate over those paths, with a wider standard error.
The per-rank solves use the FP64 oracle."""
import datetime
import multiprocessing as mproc
import os
import socket

import numpy as np
import torch

from paper_1705_03666_gb300 import shard, workloads as W

N_PATHS = 600
WORLD = 3
DEADLINE_S = 5.0


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem():
    w = W.workload(2)
    return w, w["nodes"][::256]


def _solve(oracle, w, nodes, lo, hi, p_lo, p_hi):
    r = oracle.interface_solve(w["prob"], nodes[lo:hi], node_ids=np.arange(lo, hi),
                               seed=w["seed"], dt=1e-3, n_paths=p_hi - p_lo, path_offset=p_lo,
                               n_threads=1)
    return shard.triples(torch.from_numpy(r["mean"]), torch.from_numpy(r["se"]),
                         torch.from_numpy(r["n"]))


def _worker(rank, port, mode, fail_rank, out_dir, late=None):
    """late = (late_rank, slow_rank): late_rank publishes just after the
    first deadline, and slow_rank starts collecting later, so that one
    survivor sees the late table and another does not."""
    import time

    import torch.distributed as dist

    import oracle
    w, nodes = _problem()
    n = len(nodes)
    store = dist.TCPStore("127.0.0.1", port, WORLD, rank == 0,
                          datetime.timedelta(seconds=60))
    if mode == "nodes":
        lo, hi = shard.node_block(n, WORLD, rank)
        t = _solve(oracle, w, nodes, lo, hi, 0, N_PATHS)
    else:
        p_lo, p_hi = shard.path_block(N_PATHS, WORLD, rank)
        t = _solve(oracle, w, nodes, 0, n, p_lo, p_hi)
    if rank == fail_rank:
        raise RuntimeError("injected failure: this rank leaves before publishing")
    if late is not None:   # start the exchange together, so the delays are what differ
        store.set(f"ready/{rank}", b"1")
        store.wait([f"ready/{r}" for r in range(WORLD)], datetime.timedelta(seconds=60))
    if late is not None and rank == late[0]:
        time.sleep(DEADLINE_S + 1.0)          # misses the first deadline
    shard.publish(store, "stage1", rank, t)
    if late is not None and rank == late[1]:
        time.sleep(2.0)                       # its deadline ends later: sees the late table
    got, lost = shard.collect(store, "stage1", range(WORLD), DEADLINE_S)
    np.save(os.path.join(out_dir, f"{mode}_{rank}_seen.npy"), np.array(sorted(got), dtype=np.int64))
    got, lost, alive = shard.agree(store, "stage1", got, lost)
    if rank not in alive:
        # declared lost by the agreed view: its table is not used
        np.save(os.path.join(out_dir, f"{mode}_{rank}_declared_lost.npy"), np.array([rank]))
        shard.publish(store, "done", rank, torch.zeros((0, 3), dtype=torch.float64))
        return
    if mode == "nodes":
        pieces = shard.lost_node_share(n, WORLD, lost, alive, rank)
        parts = [_solve(oracle, w, nodes, a, b, 0, N_PATHS) for a, b in pieces]
        redo = torch.cat(parts) if parts else torch.zeros((0, 3), dtype=torch.float64)
        shard.publish(store, "stage1-redo", rank, redo)
        got2, lost2 = shard.collect(store, "stage1-redo", alive, DEADLINE_S)
        assert not lost2
        full = shard.assemble_nodes(n, WORLD, got, lost, got2)
    else:
        full = shard.merge_surviving_paths(got)
    m, se, c = shard.finalize(full)
    np.save(os.path.join(out_dir, f"{mode}_{rank}.npy"),
            torch.stack([m, se, c.double()]).numpy())
    np.save(os.path.join(out_dir, f"{mode}_{rank}_lost.npy"), np.array(lost, dtype=np.int64))
    # the store lives in rank 0: it stays until every survivor has read it
    shard.publish(store, "done", rank, torch.zeros((0, 3), dtype=torch.float64))
    if rank == 0:
        _, late = shard.collect(store, "done", alive, 30.0)
        assert not late


def _run(tmp_path, mode, fail_rank, late=None):
    ctx = mproc.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, mode, fail_rank, str(tmp_path), late))
             for r in range(WORLD)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    return codes


def test_lost_node_block_is_recomputed_by_the_survivors(tmp_path):
    import oracle
    fail = 1
    codes = _run(tmp_path, "nodes", fail)
    assert codes[fail] != 0 and all(c == 0 for r, c in enumerate(codes) if r != fail), codes
    w, nodes = _problem()
    ref = oracle.interface_solve(w["prob"], nodes, seed=w["seed"], dt=1e-3, n_paths=N_PATHS)
    for r in (0, 2):
        got = np.load(tmp_path / f"nodes_{r}.npy")
        assert list(np.load(tmp_path / f"nodes_{r}_lost.npy")) == [fail]
        np.testing.assert_allclose(got[0], ref["mean"], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(got[1], ref["se"], rtol=1e-9)
        assert np.array_equal(got[2], ref["n"].astype(np.float64))


def test_rank_publishing_at_the_deadline_gets_one_agreed_view(tmp_path):
    """Rank 2 publishes just after rank 1's deadline; rank 0 collects later
    and sees it, rank 1 does not.  Without an agreed view rank 1 would redo
    rank 2's block alone while rank 0 waited for nothing to redo.  With it,
    all ranks act on the first view written (rank 1's: rank 2 lost), the
    survivors recompute rank 2's block and reproduce the single-process
    estimate; rank 2 learns that it was declared lost."""
    import oracle
    codes = _run(tmp_path, "nodes", fail_rank=-1, late=(2, 0))
    assert all(c == 0 for c in codes), codes
    seen = {r: list(np.load(tmp_path / f"nodes_{r}_seen.npy")) for r in range(WORLD)}
    assert seen[1] == [0, 1] and seen[0] == [0, 1, 2]      # the two survivors disagreed
    assert (tmp_path / "nodes_2_declared_lost.npy").exists()
    w, nodes = _problem()
    ref = oracle.interface_solve(w["prob"], nodes, seed=w["seed"], dt=1e-3, n_paths=N_PATHS)
    for r in (0, 1):
        got = np.load(tmp_path / f"nodes_{r}.npy")
        assert list(np.load(tmp_path / f"nodes_{r}_lost.npy")) == [2]
        np.testing.assert_allclose(got[0], ref["mean"], rtol=1e-12, atol=1e-14)
        assert np.array_equal(got[2], ref["n"].astype(np.float64))


def test_lost_path_range_only_loses_samples(tmp_path):
    import oracle
    fail = WORLD - 1
    codes = _run(tmp_path, "paths", fail)
    assert codes[fail] != 0 and all(c == 0 for r, c in enumerate(codes) if r != fail), codes
    w, nodes = _problem()
    kept = shard.path_block(N_PATHS, WORLD, fail)[0]      # survivors hold paths [0, kept)
    part = oracle.interface_solve(w["prob"], nodes, seed=w["seed"], dt=1e-3, n_paths=kept)
    full = oracle.interface_solve(w["prob"], nodes, seed=w["seed"], dt=1e-3, n_paths=N_PATHS)
    for r in range(WORLD - 1):
        got = np.load(tmp_path / f"paths_{r}.npy")
        assert list(np.load(tmp_path / f"paths_{r}_lost.npy")) == [fail]
        np.testing.assert_allclose(got[0], part["mean"], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(got[1], part["se"], rtol=1e-9)
        assert np.all(got[2] == kept)
    # fewer samples, wider error: about sqrt(600 / 400) = 1.22
    ratio = np.median(part["se"] / full["se"])
    assert 1.1 < ratio < 1.35, ratio


def test_store_exchange_helpers_on_one_process():
    store = torch.distributed.HashStore()
    a = torch.tensor([[2.0, 1.0, 0.5], [3.0, -1.0, 2.0]], dtype=torch.float64)
    shard.publish(store, "t", 0, a)
    got, lost = shard.collect(store, "t", [0, 1], timeout_s=0.05)
    assert lost == [1] and torch.equal(got[0], a)
    # node blocks: rank 1 of 3 lost, its block split over ranks 0 and 2
    n, world = 10, 3
    pieces = {r: shard.lost_node_share(n, world, [1], [0, 2], r) for r in (0, 2)}
    assert pieces == {0: [(4, 6)], 2: [(6, 7)]}
    blocks = {r: torch.full((shard.node_block(n, world, r)[1] - shard.node_block(n, world, r)[0], 3),
                            float(r)) for r in (0, 2)}
    redo = {0: torch.full((2, 3), 10.0), 2: torch.full((1, 3), 12.0)}
    t = shard.assemble_nodes(n, world, blocks, [1], redo)
    assert t[:, 0].tolist() == [0, 0, 0, 0, 10, 10, 12, 2, 2, 2]
    t0 = shard.assemble_nodes(n, world, blocks)            # nobody redid the block
    assert t0[4:7, 0].tolist() == [0, 0, 0]
    m, se, c = shard.finalize(t0)
    assert c[4:7].tolist() == [0, 0, 0]
    assert torch.isnan(m[4:7]).all() and torch.isnan(se[4:7]).all()   # no estimate there
    # an empty side never enters the merge, even with a NaN mean
    e = torch.tensor([[0.0, float("nan"), 0.0], [2.0, 1.0, 0.5]], dtype=torch.float64)
    f = torch.tensor([[3.0, 2.0, 1.0], [0.0, float("nan"), 0.0]], dtype=torch.float64)
    mg = shard.chan_merge(e, f)
    assert torch.equal(mg, torch.tensor([[3.0, 2.0, 1.0], [2.0, 1.0, 0.5]], dtype=torch.float64))
    # the agreed view: the first writer wins, later callers adopt it and read
    # the tables they missed from the store
    st = torch.distributed.HashStore()
    shard.publish(st, "v", 0, a)
    shard.publish(st, "v", 2, a)
    g1, l1, al1 = shard.agree(st, "v", {0: a, 2: a}, [1])
    g2, l2, al2 = shard.agree(st, "v", {0: a}, [1, 2])
    assert al1 == al2 == [0, 2] and l1 == l2 == [1] and sorted(g2) == [0, 2]
