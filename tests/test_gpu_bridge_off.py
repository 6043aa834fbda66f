"""GPU parity with the Brownian-bridge exit test switched off (Sec. 2.1 with
exits only where a step leaves the closed domain), against the FP64 oracle
on shared streams, for every kernel that screens its steps: the box in 2-D
and 3-D, the L-shape, reflecting faces and the batch.  With the bridge off
the step kernels keep their screening branch but its bound is identically
zero, so only the outside test can end a path.

On shared streams a path is the same random path with the bridge on and off
until the first bridge crossing, so its exit step with the bridge off is
never earlier: checked path by path.
"""
import numpy as np
import pytest
import torch

from paper_1705_03666_gb300 import workloads as W

pytestmark = pytest.mark.gpu

from tests import parity

FLIP_MAX_FP32 = 2e-4   # measured on GB300: no flips in these cases


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1705_03666_gb300 import api as a
    assert torch.cuda.is_available()
    return a


def _check(name, g, o, geometry, prob, flip_max, path_tol=None):
    c = parity.compare_paths(g, o, path_tol=path_tol, prob=prob, geometry=geometry)
    parity.check(name, c, flip_max=flip_max)


def _solve(api, prob, nodes, **kw):
    with api.Context(prob) as ctx:
        return ctx.interface_solve(torch.from_numpy(nodes), dump_paths=True, diag=True, **kw)


GEOM = {"cube": "unit_cube", "square": "unit_square", "lshape": "l_shape", "robin": "unit_square"}
CASES = {
    "cube": (W.elliptic_manufactured(), W.workload(2)["nodes"][::256], 1e-3),
    "square": (W.laplace_expcos(), W.nodes_cfg1(16), 1e-3),
    "lshape": (W.laplace_expcos("l_shape"), W.nodes_lshape_interfaces(24), 1e-3),
    "robin": (W.laplace_expcos(reflect=[1, 2], phi=-2.0), W.nodes_cfg1(16), 1e-3),
}


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_matches_oracle_without_bridge(api, orc, name):
    prob, nodes, dt = CASES[name]
    kw = dict(seed=W.SEED_BASE + 41, dt=dt, n_paths=1500, bridge=False)
    g = _solve(api, prob, nodes, precision="fp32", **kw)
    o = orc.interface_solve(prob, nodes, dump_paths=True, **kw)
    _check(f"bridge off {name} fp32", g, o, GEOM[name], prob, FLIP_MAX_FP32)
    assert g["capped"] == 0


@pytest.mark.parametrize("name", ["cube", "lshape"])
def test_fp64_matches_oracle_without_bridge(api, orc, name):
    prob, nodes, dt = CASES[name]
    kw = dict(seed=W.SEED_BASE + 42, dt=dt, n_paths=500, bridge=False)
    g = _solve(api, prob, nodes, precision="fp64", **kw)
    o = orc.interface_solve(prob, nodes, dump_paths=True, **kw)
    _check(f"bridge off {name} fp64", g, o, GEOM[name], None, 1e-4, path_tol=1e-11)
    np.testing.assert_allclose(g["mean"].cpu().numpy(), o["mean"], rtol=1e-9)


@pytest.mark.parametrize("name", list(CASES))
def test_exit_never_earlier_without_bridge(api, name):
    prob, nodes, dt = CASES[name]
    kw = dict(seed=W.SEED_BASE + 43, dt=dt, n_paths=2000, precision="fp32")
    on = _solve(api, prob, nodes, bridge=True, **kw)["steps"].cpu().numpy()
    off = _solve(api, prob, nodes, bridge=False, **kw)["steps"].cpu().numpy()
    assert np.all(off >= on)
    assert (off > on).mean() > 0.05     # the bridge ends a fair share of paths earlier


def test_batch_matches_interface_solve_without_bridge(api):
    """The batch's per-family kernels with the bridge off run the same paths
    as pdd_interface_solve: equal step totals, means to reduction rounding."""
    prob, nodes, dt = CASES["lshape"]
    n, N = len(nodes), 3000
    nodes3 = np.zeros((n, 3))
    nodes3[:, :2] = nodes
    with api.Context(prob) as ctx:
        r = ctx.batch_solve([prob], torch.from_numpy(nodes3), torch.zeros(n, dtype=torch.int32),
                            torch.full((n,), dt, dtype=torch.float64), seed=5, n_pilot=300,
                            n_min=N, n_max=N, target_se=1.0, bridge=False, diag=True)
        p = ctx.interface_solve(torch.from_numpy(nodes), seed=5, dt=dt, n_paths=N,
                                precision="fp32", bridge=False, diag=True)
    assert r["path_steps"] == p["path_steps"]
    np.testing.assert_allclose(r["mean"].cpu().numpy(), p["mean"].cpu().numpy(), rtol=1e-9,
                               atol=1e-12)
