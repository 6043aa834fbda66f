"""Checkpoint / resume of an interface solve (host logic, CPU): a run split
into pieces, stopped and resumed from the file, gives the single run's
estimate (same paths by path_offset; Chan merge of the triples); a
checkpoint refuses other settings.  The solves here are the FP64 oracle's."""
import numpy as np
import pytest

from paper_1705_03666_gb300 import checkpoint as C, workloads as W


def _oracle_solve(orc, prob, calls):
    def solve(nodes, *, seed, dt, n_paths, path_offset, precision, bridge, max_steps):
        calls.append((path_offset, n_paths))
        return orc.interface_solve(prob, nodes, seed=seed, dt=dt, n_paths=n_paths,
                                   path_offset=path_offset, bridge=bridge,
                                   max_steps=max_steps, n_threads=2)
    return solve


def _setup():
    w = W.workload(2)
    return w["prob"], w["nodes"][::512], dict(seed=w["seed"], dt=2e-3, precision="fp64")


def test_pieces_and_resume_equal_one_run(orc, tmp_path):
    prob, nodes, run = _setup()
    ref = orc.interface_solve(prob, nodes, seed=run["seed"], dt=run["dt"], n_paths=700)
    calls = []
    solve = _oracle_solve(orc, prob, calls)
    path = str(tmp_path / "ck.npz")
    # first session: 300 paths in pieces of 128, then it stops
    r1 = C.solve_resumable(solve, prob, nodes, n_paths=300, piece=128, path=path, **run)
    assert calls == [(0, 128), (128, 128), (256, 44)]
    assert r1["next_path"] == 300 and np.all(r1["n"] == 300)
    # second session resumes from the file up to 700
    calls.clear()
    r2 = C.solve_resumable(solve, prob, nodes, n_paths=700, piece=250, path=path, **run)
    assert calls == [(300, 250), (550, 150)]
    np.testing.assert_allclose(r2["mean"], ref["mean"], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(r2["se"], ref["se"], rtol=1e-9)
    assert np.array_equal(r2["n"], ref["n"])
    # a finished checkpoint runs nothing more
    calls.clear()
    r3 = C.solve_resumable(solve, prob, nodes, n_paths=700, piece=250, path=path, **run)
    assert calls == [] and np.array_equal(r3["mean"], r2["mean"])
    with pytest.raises(ValueError, match="already holds"):
        C.solve_resumable(solve, prob, nodes, n_paths=600, piece=250, path=path, **run)


def test_checkpoint_refuses_other_settings(orc, tmp_path):
    prob, nodes, run = _setup()
    path = str(tmp_path / "ck.npz")
    solve = _oracle_solve(orc, prob, [])
    C.solve_resumable(solve, prob, nodes, n_paths=64, piece=64, path=path, **run)
    other = [dict(run, seed=run["seed"] + 1), dict(run, dt=1e-3), dict(run, precision="fp32"),
             dict(run, bridge=False), dict(run, max_steps=1000)]
    for r in other:
        with pytest.raises(ValueError, match="another problem"):
            C.solve_resumable(solve, prob, nodes, n_paths=128, piece=64, path=path, **r)
    moved = nodes.copy()
    moved[0, 0] += 1e-12
    with pytest.raises(ValueError, match="another problem"):
        C.solve_resumable(solve, prob, moved, n_paths=128, piece=64, path=path, **run)
    with pytest.raises(ValueError, match="another problem"):
        C.solve_resumable(solve, dict(prob, sigma=0.9), nodes, n_paths=128, piece=64,
                          path=path, **run)


def test_save_load_round_trip(tmp_path):
    prob, nodes, run = _setup()
    ck = C.Checkpoint.start(prob, nodes, **run)
    ck.add({"mean": np.arange(len(nodes), dtype=float), "se": np.full(len(nodes), 0.5),
            "n": np.full(len(nodes), 10)}, 10)
    p = str(tmp_path / "a.npz")
    ck.save(p)
    back = C.Checkpoint.load(p)
    assert back.digest == ck.digest and back.next_path == 10
    assert np.array_equal(back.table.numpy(), ck.table.numpy())
    r = back.result()
    np.testing.assert_allclose(r["se"], 0.5, rtol=1e-14)
    with pytest.raises(ValueError):
        ck.add({"mean": np.zeros(1), "se": np.zeros(1), "n": np.ones(1)}, 1)


def test_truncated_checkpoint_gives_a_clear_error(orc, tmp_path):
    prob, nodes, run = _setup()
    path = str(tmp_path / "ck.npz")
    C.solve_resumable(_oracle_solve(orc, prob, []), prob, nodes, n_paths=200, piece=100,
                      path=path, **run)
    raw = open(path, "rb").read()
    for cut in (0, 10, len(raw) // 2):
        with open(path, "wb") as f:
            f.write(raw[:cut])
        with pytest.raises(ValueError, match="unreadable"):
            C.Checkpoint.load(path)
        with pytest.raises(ValueError, match="unreadable"):
            C.solve_resumable(_oracle_solve(orc, prob, []), prob, nodes, n_paths=300, piece=100,
                              path=path, **run)
