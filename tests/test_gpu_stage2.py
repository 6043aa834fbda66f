"""GPU checks of stage two (Sec. 2.1): interface spline + subdomain solve,
against the oracle's SciPy spline and sparse direct solve of the same 5-point
system, and the whole two-stage PDD of the 2-D Laplace workload against the
exact harmonic solution."""
import numpy as np
import pytest
import torch

from paper_1705_03666_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1705_03666_gb300 import api as a
    return a


def _oracle_subdomain(orc, lo, hi, n, side, s_nodes, vals):
    nx, ny = n
    x = np.linspace(lo[0], hi[0], nx)
    y = np.linspace(lo[1], hi[1], ny)
    X, Y = np.meshgrid(x, y)
    u = np.exp(X) * np.cos(Y)
    u[1:-1, 1:-1] = 0.0
    col = nx - 1 if side else 0
    xf = x[col]
    u[:, col] = orc.spline_interface(s_nodes, vals, y, np.exp(xf) * np.cos(lo[1]),
                                     np.exp(xf) * np.cos(hi[1]), lo[1], hi[1])
    return orc.stencil_solve(u, ((hi[0] - lo[0]) / (nx - 1), (hi[1] - lo[1]) / (ny - 1)))


@pytest.mark.parametrize("method", ["cg", "cg_mixed"])
@pytest.mark.parametrize("side,lo,hi", [(1, (0.0, 0.0), (0.5, 1.0)), (0, (0.5, 0.0), (1.0, 1.0))])
def test_cg_matches_direct_solve(api, orc, side, lo, hi, method):
    s = W.nodes_cfg1(16)[:, 1]
    rng = np.random.default_rng(3)
    vals = np.exp(0.5) * np.cos(s) + 1e-3 * rng.standard_normal(16)   # noisy MC-like data
    with api.Context(W.laplace_expcos()) as ctx:
        r = ctx.subdomain_solve(lo, hi, (129, 129), 0, side, torch.from_numpy(s),
                                torch.from_numpy(vals), method=method, tol=1e-13)
    ref = _oracle_subdomain(orc, lo, hi, (129, 129), side, s, vals)
    assert r["status"] == 0 and r["resid"] <= 1e-13
    assert np.max(np.abs(r["u"].cpu().numpy() - ref)) < 1e-10


@pytest.mark.parametrize("n", [(37, 45), (9, 5), (200, 9)])
def test_cg_on_ragged_grids(api, orc, n):
    """FP64 CG on grids whose rows split unevenly over the blocks of the
    solve's cluster (45 and 9 rows over 8 blocks), and on a grid with fewer
    rows than blocks (one block)."""
    s = np.array([0.15, 0.4, 0.55, 0.85])
    vals = np.exp(0.5) * np.cos(s)
    with api.Context(W.laplace_expcos()) as ctx:
        r = ctx.subdomain_solve((0.0, 0.0), (0.5, 1.0), n, 0, 1, torch.from_numpy(s),
                                torch.from_numpy(vals), method="cg", tol=1e-13)
    ref = _oracle_subdomain(orc, (0.0, 0.0), (0.5, 1.0), n, 1, s, vals)
    assert r["status"] == 0 and r["resid"] <= 1e-13
    assert np.max(np.abs(r["u"].cpu().numpy() - ref)) < 1e-10


def test_jacobi_matches_direct_solve(api, orc):
    s = np.array([0.2, 0.45, 0.6, 0.9])
    vals = np.exp(0.5) * np.cos(s)
    with api.Context(W.laplace_expcos()) as ctx:
        r = ctx.subdomain_solve((0.0, 0.0), (0.5, 1.0), (17, 33), 0, 1, torch.from_numpy(s),
                                torch.from_numpy(vals), method="jacobi", tol=1e-14,
                                max_iter=200000)
    ref = _oracle_subdomain(orc, (0.0, 0.0), (0.5, 1.0), (17, 33), 1, s, vals)
    assert r["status"] == 0
    assert np.max(np.abs(r["u"].cpu().numpy() - ref)) < 1e-10


def test_iteration_cap_reported(api):
    s = np.array([0.3, 0.6, 0.8])
    with api.Context(W.laplace_expcos()) as ctx:
        r = ctx.subdomain_solve((0.0, 0.0), (0.5, 1.0), (65, 65), 0, 1, torch.from_numpy(s),
                                torch.from_numpy(np.cos(s)), method="jacobi", tol=0.0,
                                max_iter=10)
    assert r["status"] == 4 and r["iters"] == 10


def test_two_stage_pdd_laplace(api):
    """Stage one (16 nodes, 1e4 FP64 paths, dt = 1e-3) then stage two on both
    subdomains (129 x 129, CG): error of the glued solution against e^x cos y
    is at the Monte Carlo level."""
    w = W.workload(1)
    with api.Context(w["prob"]) as ctx:
        r = ctx.interface_solve(torch.from_numpy(w["nodes"]), seed=w["seed"], dt=w["dt"],
                                n_paths=w["n_paths"], precision="fp64")
        s = torch.from_numpy(w["nodes"][:, 1])
        left = ctx.subdomain_solve((0.0, 0.0), (0.5, 1.0), (129, 129), 0, 1, s, r["mean"])
        right = ctx.subdomain_solve((0.5, 0.0), (1.0, 1.0), (129, 129), 0, 0, s, r["mean"])
    se_max = float(r["se"].max())
    for part, (x0, x1) in ((left, (0.0, 0.5)), (right, (0.5, 1.0))):
        x = np.linspace(x0, x1, 129)
        y = np.linspace(0.0, 1.0, 129)
        X, Y = np.meshgrid(x, y)
        err = np.max(np.abs(part["u"].cpu().numpy() - np.exp(X) * np.cos(Y)))
        assert part["status"] == 0
        assert err < 4.0 * se_max + 1e-3, err


def test_mixed_cg_on_an_anisotropic_and_ragged_grid(api, orc):
    """FP32 CG inside FP64 refinement reaches the FP64 answer on a grid
    whose sizes are not multiples of the block (97 x 201, hx != hy)."""
    s = np.linspace(0.05, 0.95, 9)
    vals = np.exp(0.5) * np.cos(s)
    lo, hi = (0.0, 0.0), (0.5, 1.0)
    with api.Context(W.laplace_expcos()) as ctx:
        r = ctx.subdomain_solve(lo, hi, (97, 201), 0, 1, torch.from_numpy(s),
                                torch.from_numpy(vals), method="cg_mixed", tol=1e-12)
    ref = _oracle_subdomain(orc, lo, hi, (97, 201), 1, s, vals)
    assert r["status"] == 0 and r["resid"] <= 1e-12
    assert np.max(np.abs(r["u"].cpu().numpy() - ref)) < 1e-9


def test_two_stage_pdd_solve_end_to_end(api, orc):
    """Stage one (16 interface nodes, FP64 paths) then stage two (spline +
    both halves).  By the discrete maximum principle, the error of each half
    is bounded by its boundary error -- on the interface, the spline of the
    Monte Carlo values against e^x cos y -- plus the O(h^2) consistency error
    of the 5-point scheme."""
    prob = W.laplace_expcos()
    with api.Context(prob) as ctx:
        r = api.laplace_pdd_solve(ctx, n_paths=40_000, seed=W.SEED_BASE + 51)
    assert r["status"] == 0
    ny, nx = r["left"].shape
    ys = np.linspace(0.0, 1.0, ny)
    s = r["nodes"][:, 1].numpy()
    spl = orc.spline_interface(s, r["mean"].cpu().numpy(), ys, np.exp(0.5), np.exp(0.5) * np.cos(1.0))
    iface_err = np.max(np.abs(spl - np.exp(0.5) * np.cos(ys)))
    for u, x0 in ((r["left"], 0.0), (r["right"], 0.5)):
        X, Y = np.meshgrid(np.linspace(x0, x0 + 0.5, nx), ys)
        err = np.max(np.abs(u.cpu().numpy() - np.exp(X) * np.cos(Y)))
        assert err <= iface_err + 2e-5, (err, iface_err)
    # the interface column of both halves is the same spline
    assert torch.allclose(r["left"][:, -1], r["right"][:, 0], rtol=0, atol=1e-14)
    # and the Monte Carlo node values are within their standard errors
    exact = np.exp(0.5) * np.cos(s)
    assert np.all(np.abs(r["mean"].cpu().numpy() - exact) <= 4.5 * r["se"].cpu().numpy() + 2e-3)


@pytest.mark.parametrize("side,lo,hi", [(1, (0.0, 0.0), (0.5, 1.0)), (0, (0.5, 0.0), (1.0, 1.0))])
def test_dst_matches_direct_solve(api, orc, side, lo, hi):
    """The sine-transform solve is the discrete solution itself: against the
    oracle's sparse direct solve and the FP64 CG on the same data."""
    s = W.nodes_cfg1(16)[:, 1]
    rng = np.random.default_rng(5)
    vals = np.exp(0.5) * np.cos(s) + 1e-3 * rng.standard_normal(16)
    with api.Context(W.laplace_expcos()) as ctx:
        r = ctx.subdomain_solve(lo, hi, (129, 129), 0, side, torch.from_numpy(s),
                                torch.from_numpy(vals), method="dst")
        c = ctx.subdomain_solve(lo, hi, (129, 129), 0, side, torch.from_numpy(s),
                                torch.from_numpy(vals), method="cg", tol=1e-14)
    ref = _oracle_subdomain(orc, lo, hi, (129, 129), side, s, vals)
    assert r["status"] == 0 and r["iters"] == 0 and r["resid"] <= 1e-12, r["resid"]
    assert np.max(np.abs(r["u"].cpu().numpy() - ref)) < 1e-11
    assert float((r["u"] - c["u"]).abs().max()) < 1e-10


@pytest.mark.parametrize("n", [(97, 201), (3, 3), (3, 40), (40, 3), (4, 5)])
def test_dst_on_anisotropic_ragged_and_degenerate_grids(api, orc, n):
    """Grid sizes not multiples of the 32-point tiles, hx != hy, and one
    interior point per axis."""
    s = np.linspace(0.05, 0.95, 9)
    vals = np.exp(0.5) * np.cos(s)
    lo, hi = (0.0, 0.0), (0.5, 1.0)
    with api.Context(W.laplace_expcos()) as ctx:
        r = ctx.subdomain_solve(lo, hi, n, 0, 1, torch.from_numpy(s), torch.from_numpy(vals),
                                method="dst")
    ref = _oracle_subdomain(orc, lo, hi, n, 1, s, vals)
    assert r["status"] == 0 and r["resid"] <= 1e-12, r["resid"]
    assert np.max(np.abs(r["u"].cpu().numpy() - ref)) < 1e-11


def test_dst_limits_and_dirichlet_only_data(api):
    """Axes beyond 8192 interior points are refused (EINVAL, before any
    allocation); on a small ragged grid the interior of the direct solution
    obeys the discrete maximum principle."""
    from paper_1705_03666_gb300._lib import PDDError
    s = np.array([0.25, 0.5, 0.75])
    with api.Context(W.laplace_expcos()) as ctx:
        with pytest.raises(PDDError):
            ctx.subdomain_solve((0.0, 0.0), (0.5, 1.0), (8195, 3), 0, 1, torch.from_numpy(s),
                                torch.from_numpy(np.zeros(3)), method="dst")
        r = ctx.subdomain_solve((0.0, 0.0), (0.5, 1.0), (33, 17), 0, 1, torch.from_numpy(s),
                                torch.from_numpy(np.exp(0.5) * np.cos(s)), method="dst")
    assert r["status"] == 0 and r["iters"] == 0
    u = r["u"].cpu().numpy()
    assert np.all(np.isfinite(u))
    # discrete maximum principle: the interior lies within the boundary's range
    bd = np.concatenate([u[0], u[-1], u[:, 0], u[:, -1]])
    assert u[1:-1, 1:-1].max() <= bd.max() + 1e-12 and u[1:-1, 1:-1].min() >= bd.min() - 1e-12
