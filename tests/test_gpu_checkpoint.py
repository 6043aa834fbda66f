"""Resume of a GPU interface solve by path_offset: the paths of a call with
path_offset k are paths k.. of a call without it, bit for bit, and a run
checkpointed in pieces through a file gives the one-call estimate."""
import numpy as np
import pytest
import torch

from paper_1705_03666_gb300 import checkpoint as C, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1705_03666_gb300 import api as a
    assert torch.cuda.is_available()
    return a


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_resume_by_path_offset_reproduces_one_run(api, tmp_path, precision):
    w = W.workload(2)
    nodes = torch.from_numpy(np.ascontiguousarray(w["nodes"][::64]))
    run = dict(seed=w["seed"], dt=1e-3, precision=precision)
    with api.Context(w["prob"], 0) as ctx:
        full = ctx.interface_solve(nodes, n_paths=2000, dump_paths=True, **run)
        part = ctx.interface_solve(nodes, n_paths=1200, path_offset=800, dump_paths=True, **run)
        torch.cuda.synchronize()
        assert torch.equal(part["score"], full["score"][:, 800:])
        assert torch.equal(part["steps"], full["steps"][:, 800:])

        def solve(nodes_, *, n_paths, path_offset, **kw):
            return ctx.interface_solve(nodes_, n_paths=n_paths, path_offset=path_offset, **kw)

        path = str(tmp_path / "ck.npz")
        C.solve_resumable(solve, w["prob"], nodes, n_paths=900, piece=700, path=path, **run)
        r = C.solve_resumable(solve, w["prob"], nodes, n_paths=2000, piece=700, path=path, **run)
    assert r["next_path"] == 2000
    np.testing.assert_allclose(r["mean"], full["mean"].cpu().numpy(), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(r["se"], full["se"].cpu().numpy(), rtol=1e-9)
    assert np.array_equal(r["n"], full["n"].cpu().numpy())
