"""GPU parity of reflecting (Neumann/Robin) faces against the FP64 oracle:
the mixed BVP of Eq. 2.4 through the local-time system of Eq. 2.9 with
Lepingle's half-space reflection, on shared Philox streams (the step's
stream as for absorbing paths, the reflection uniforms from tag 4)."""
import numpy as np
import pytest
import torch

from paper_1705_03666_gb300 import workloads as W

pytestmark = pytest.mark.gpu

from tests import parity


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1705_03666_gb300 import api as a
    assert torch.cuda.is_available()
    return a


def _parity(api, orc, prob, nodes, precision, flip_max, tol, **kw):
    o = orc.interface_solve(prob, nodes, dump_paths=True, **kw)
    with api.Context(prob) as ctx:
        g = ctx.interface_solve(torch.from_numpy(nodes), precision=precision, dump_paths=True,
                                diag=True, **kw)
    if precision == "fp32":
        c = parity.compare_paths(g, o, prob=prob, geometry=prob["geometry"])
    else:
        c = parity.compare_paths(g, o, path_tol=tol, geometry=prob["geometry"])
    faces = "".join(str(int(v)) for v in prob["params"][:1])
    parity.check(f"reflecting mask {faces} {prob['problem']} {precision}", c, flip_max=flip_max)
    return g, o


LAPLACE_NODES = np.array([[0.5, 0.5], [0.9, 0.2], [0.3, 0.05], [0.5, 0.0], [0.95, 0.9], [0.02, 0.5]])


@pytest.mark.parametrize("reflect,phi", [([2], 0.0), ([1, 2], -2.0), ([0, 1, 2], -0.5)])
def test_laplace_fp64_path_by_path(api, orc, reflect, phi):
    prob = W.laplace_expcos(reflect=reflect, phi=phi)
    g, o = _parity(api, orc, prob, LAPLACE_NODES, "fp64", 1e-4, 1e-9, seed=W.SEED_BASE + 31,
                   dt=1e-3, n_paths=2000)
    assert g["path_steps"] > 0


@pytest.mark.parametrize("reflect,phi", [([2], 0.0), ([1, 2], -2.0)])
def test_laplace_fp32(api, orc, reflect, phi):
    prob = W.laplace_expcos(reflect=reflect, phi=phi)
    _parity(api, orc, prob, LAPLACE_NODES, "fp32", 2e-4, None, seed=W.SEED_BASE + 32, dt=1e-3,
            n_paths=3000)


def test_elliptic_3d_robin_fp32_and_fp64(api, orc):
    prob = W.elliptic_manufactured(reflect=[4, 0], phi=-1.0)
    nodes = np.array([[0.5, 0.5, 0.1], [0.1, 0.5, 0.5], [0.3, 0.7, 0.25], [0.0, 0.4, 0.6]])
    _parity(api, orc, prob, nodes, "fp32", 2e-4, None, seed=W.SEED_BASE + 33, dt=1e-3, n_paths=2000)
    _parity(api, orc, prob, nodes, "fp64", 1e-4, 1e-9, seed=W.SEED_BASE + 34, dt=1e-3, n_paths=1000)


def test_closed_form_at_size(api):
    """16 nodes x 2e5 paths: e^x cos y with Neumann y = 0 and Robin x = 1
    (phi = -2) within 4.5 sigma plus an O(dt) allowance."""
    prob = W.laplace_expcos(reflect=[1, 2], phi=-2.0)
    nodes = np.stack([np.linspace(0.05, 0.95, 16), np.linspace(0.0, 0.9, 16)], 1)
    with api.Context(prob) as ctx:
        r = ctx.interface_solve(torch.from_numpy(nodes), seed=W.SEED_BASE + 35, dt=1e-3,
                                n_paths=200_000, precision="fp32", diag=True)
    exact = np.exp(nodes[:, 0]) * np.cos(nodes[:, 1])
    m, se = r["mean"].cpu().numpy(), r["se"].cpu().numpy()
    assert np.all(np.abs(m - exact) <= 4.5 * se + 2e-3), (m - exact) / se
    assert r["capped"] == 0


def test_rejections(api):
    with pytest.raises(Exception):
        api.Context(W.laplace_expcos("l_shape", reflect=[1]))
    bad = W.laplace_expcos(reflect=[1], phi=0.5)
    with pytest.raises(Exception):
        api.Context(bad)
    bad = W.laplace_expcos()
    bad["params"] = np.array([99.0, 0.0])
    with pytest.raises(Exception):
        api.Context(bad)
    with api.Context(W.laplace_expcos(reflect=[2])) as ctx:
        with pytest.raises(Exception):
            ctx.wos_solve(torch.tensor([[0.5, 0.5]]), seed=1, n_paths=8, eps=1e-3)
        with pytest.raises(Exception):
            ctx.interface_solve_naive(torch.tensor([[0.5, 0.5]]), seed=1, dt=1e-3, n_paths=8)
