"""GPU parity of pdd_interface_solve against the FP64 oracle (shared streams).

Both sides consume the same Philox4x32-10 words, so every path is the same
random path.  The FP64 path kernel must reproduce the oracle's exit steps and
scores to rounding.  The FP32 path kernel differs from FP64 by rounding of the
position, so a rare path takes its exit decision at a different step or
through a different face (an exit flip); flips are counted, reported and must
stay near their measured rate, no path that exits at the same step through the
same face may differ from the oracle beyond the per-path bound, and the node
means over those paths must agree to 1e-5 relative (tests/parity.py).
Full-size runs are checked on sampled nodes and against the closed-form
solution.
"""
import numpy as np
import pytest
import torch

from paper_1705_03666_gb300 import workloads as W
from tests import parity

pytestmark = pytest.mark.gpu

# Binary32 paths that exit at the same step through the same face as the
# binary64 oracle must stay within the per-path bound of tests/parity.py
# (exit-point rounding times |grad g|).  Exit-flip limit: the fractions
# measured on GB300 are 0 to 4e-5 (printed by every run; 3.7e-5 on the
# full-size workload's sampled nodes), the limit a few times that.
FLIP_MAX_FP32 = 2e-4
NODE_REL_TOL = parity.NODE_REL_TOL


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1705_03666_gb300 import api as a
    assert torch.cuda.is_available()
    return a


def test_philox_bit_exact(api, orc):
    cases = [(W.SEED_BASE + 2, 0, 5, 7, 0, 1 << 20),
             (0, 2 ** 32 - 1000, 2 ** 32 - 1, 0, 1, 4096),
             (2 ** 64 - 1, 123, 0, 4095, 0, 4096)]
    with api.Context(W.laplace_expcos()) as ctx:
        for seed, j0, c1, c2, c3, nb in cases:
            g = ctx.philox_stream(seed, j0, c1, c2, c3, nb).cpu().numpy().view(np.uint32)
            o = orc.philox_stream(seed, j0, c1, c2, c3, nb)
            assert np.array_equal(g, o), (seed, j0, c1, c2, c3)


def test_fp32_normals_match_oracle(api, orc):
    """The binary32 Box-Muller normals (hardware log2 for -2 ln u, hardware
    sin/cos on a centred angle) against the oracle's FP64 normals from the
    same words.  Error model: the hardware log2 has an absolute error of order
    2^-22, so r^2 = -2 ln u carries ~2e-7 absolute and r = sqrt(r^2) carries
    ~1e-7 / r; sin/cos add ~4e-7 r; rounding ~1e-7 |z|.  The bound below is
    that model with a safety factor; it is loose only for the rare pairs
    with a tiny radius (a 1e-3 radius has probability 5e-7)."""
    n = 1 << 22
    with api.Context(W.laplace_expcos()) as ctx:
        z, u = ctx.normals(W.SEED_BASE + 7, n, 3, 4, 9)
    zo, uo = orc.normals(W.SEED_BASE + 7, n, 3, 4, 9)
    z, u = z.cpu().numpy().astype(np.float64), u.cpu().numpy().astype(np.float64)
    assert np.array_equal(u, uo)                               # exact uniforms
    err = np.abs(z - zo)
    r = np.repeat(np.hypot(zo[0::2], zo[1::2]), 2)
    bound = 4e-7 / np.maximum(r, 1e-4) + 2e-6 * np.maximum(1.0, np.abs(zo))
    assert np.all(err <= bound), (err / bound).max()
    assert np.mean(err) < 5e-7
    # away from tiny radii the normals are accurate to a few 1e-7
    big = r > 0.5
    assert np.max(err[big] / np.maximum(1.0, np.abs(zo[big]))) < 2e-6


def test_laplace_fp64_matches_oracle_path_by_path(api, orc):
    w = W.workload(1)
    kw = dict(seed=w["seed"], dt=w["dt"], n_paths=4000)
    with api.Context(w["prob"]) as ctx:
        g = ctx.interface_solve(torch.from_numpy(w["nodes"]), precision="fp64", dump_paths=True, **kw)
    o = orc.interface_solve(w["prob"], w["nodes"], dump_paths=True, **kw)
    c = parity.compare_paths(g, o, path_tol=1e-12, geometry="unit_square")
    parity.check("laplace2d fp64", c, flip_max=1e-4)
    mg = g["mean"].cpu().numpy()
    np.testing.assert_allclose(mg, o["mean"], rtol=1e-10)
    np.testing.assert_allclose(g["se"].cpu().numpy(), o["se"], rtol=1e-6)
    assert np.array_equal(g["n"].cpu().numpy(), o["n"])
    assert g["path_steps"] == o["total_steps"]


@pytest.mark.parametrize("dt,stride,n_paths", [(1e-3, 64, 3001), (1e-4, 256, 1000)])
def test_elliptic_fp32_matches_oracle(api, orc, dt, stride, n_paths):
    w = W.workload(2)
    nodes = w["nodes"][::stride]
    kw = dict(seed=w["seed"], dt=dt, n_paths=n_paths)
    with api.Context(w["prob"]) as ctx:
        g = ctx.interface_solve(torch.from_numpy(nodes), precision="fp32", dump_paths=True, **kw)
    o = orc.interface_solve(w["prob"], nodes, dump_paths=True, **kw)
    c = parity.compare_paths(g, o, prob=w["prob"], geometry="unit_cube")
    parity.check(f"elliptic3d fp32 dt={dt}", c, flip_max=FLIP_MAX_FP32)
    # the per-node statistics themselves (all paths) agree within the flips' reach
    se = o["se"]
    assert np.all(np.abs(g["mean"].cpu().numpy() - o["mean"]) <= 0.5 * se + 1e-6)


def test_elliptic_fp64_matches_oracle(api, orc):
    w = W.workload(2)
    nodes = w["nodes"][::512]
    kw = dict(seed=w["seed"], dt=1e-3, n_paths=1000)
    with api.Context(w["prob"]) as ctx:
        g = ctx.interface_solve(torch.from_numpy(nodes), precision="fp64", dump_paths=True, **kw)
    o = orc.interface_solve(w["prob"], nodes, dump_paths=True, **kw)
    c = parity.compare_paths(g, o, path_tol=1e-11, geometry="unit_cube")
    parity.check("elliptic3d fp64", c, flip_max=1e-4)
    np.testing.assert_allclose(g["mean"].cpu().numpy(), o["mean"], rtol=1e-10)


def test_poisson_fourier_fp32_matches_oracle(api, orc):
    w = W.workload(5)
    nodes = w["nodes"][::64]
    kw = dict(seed=w["seed"], dt=1e-3, n_paths=2000)
    with api.Context(w["prob"]) as ctx:
        g = ctx.interface_solve(torch.from_numpy(nodes), precision="fp32", dump_paths=True, **kw)
    o = orc.interface_solve(w["prob"], nodes, dump_paths=True, **kw)
    c = parity.compare_paths(g, o, prob=w["prob"], geometry="unit_square")
    parity.check("poisson_fourier fp32", c, flip_max=FLIP_MAX_FP32)


def test_waves_and_launch_shape_do_not_change_results(api):
    w = W.workload(2)
    nodes = torch.from_numpy(w["nodes"][::128])
    kw = dict(seed=w["seed"], dt=1e-3, n_paths=2999, precision="fp32", dump_paths=True)
    with api.Context(w["prob"]) as ctx:
        a = ctx.interface_solve(nodes, **kw)
        ctx.set_tuning(blocks_per_sm=1, wave_max_paths=10007)  # ragged waves across nodes
        b = ctx.interface_solve(nodes, **kw)
        ctx.set_tuning(0, 0)
        c = ctx.interface_solve(nodes, **kw)
    assert torch.equal(a["score"], b["score"]) and torch.equal(a["steps"], b["steps"])
    assert torch.equal(a["exit"], b["exit"])
    assert torch.equal(a["mean"], c["mean"]) and torch.equal(a["se"], c["se"])  # deterministic
    # the per-node sums are exact integers: another launch shape gives the
    # same bits, not just the same values to rounding
    assert torch.equal(a["mean"], b["mean"]) and torch.equal(a["se"], b["se"])
    assert a["path_steps"] == b["path_steps"]


def test_node_offset_reproduces_node_blocks(api):
    """A block of the node list solved on its own with node_offset = its first
    index draws the streams of the single call: bit-equal paths and means."""
    w = W.workload(2)
    nodes = w["nodes"][:96]
    kw = dict(seed=w["seed"], dt=1e-3, n_paths=700, precision="fp32", dump_paths=True)
    with api.Context(w["prob"]) as ctx:
        full = ctx.interface_solve(torch.from_numpy(nodes), **kw)
        for lo, hi in ((0, 40), (40, 41), (41, 96)):
            part = ctx.interface_solve(torch.from_numpy(nodes[lo:hi]), node_offset=lo, **kw)
            for k in ("score", "steps", "exit", "mean", "se", "n"):
                assert torch.equal(part[k], full[k][lo:hi]), (lo, k)
        shifted = ctx.interface_solve(torch.from_numpy(nodes[40:96]), **kw)
    assert not torch.equal(shifted["score"], full["score"][40:96])   # other streams


def test_edge_cases(api):
    from paper_1705_03666_gb300._lib import NODE_FLAGS as F
    w = W.workload(1)
    with api.Context(w["prob"]) as ctx:
        # empty input: nothing to do
        r = ctx.interface_solve(torch.zeros((0, 2), dtype=torch.float64), seed=1, dt=1e-3,
                                n_paths=10, diag=True)
        assert r["mean"].numel() == 0 and r["path_steps"] == 0
        # a single path of a single node
        r = ctx.interface_solve(torch.tensor([[0.5, 0.5]]), seed=1, dt=1e-3, n_paths=1, diag=True)
        assert r["n"].item() == 1 and r["se"].item() == 0.0 and r["path_steps"] > 0
        # nodes on the boundary: u = g exactly, zero error, zero steps
        bn = np.array([[0.0, 0.3], [0.5, 1.0], [1.0, 0.0]])
        r = ctx.interface_solve(torch.from_numpy(bn), seed=1, dt=1e-3, n_paths=33,
                                precision="fp64", dump_paths=True)
        g = np.exp(bn[:, 0]) * np.cos(bn[:, 1])
        np.testing.assert_allclose(r["mean"].cpu().numpy(), g, rtol=1e-15)
        assert np.all(r["se"].cpu().numpy() == 0.0)
        assert int(r["steps"].abs().sum()) == 0
        assert np.all(r["flags"].cpu().numpy() == F["on_boundary"])
        assert torch.equal(r["exit"][:, 0, :].cpu(), torch.from_numpy(bn))
        # step cap: every path capped, counted, status ECAP, node flagged
        r = ctx.interface_solve(torch.tensor([[0.5, 0.5], [0.5, 0.0]]), seed=1, dt=1e-7,
                                n_paths=100, max_steps=3, diag=True)
        assert r["status"] == 5 and r["capped"] == 100 and r["path_steps"] == 300
        assert r["flags"].cpu().tolist() == [F["capped"], F["on_boundary"]]
        # a node outside the closed domain is an invalid input: with diag the
        # call reports it; without, its mean is NaN and (with flags) flagged
        from paper_1705_03666_gb300._lib import PDDError
        with pytest.raises(PDDError):
            ctx.interface_solve(torch.tensor([[1.5, 0.5]]), seed=1, dt=1e-3, n_paths=4, diag=True)
        r = ctx.interface_solve(torch.tensor([[0.5, 0.5], [1.5, 0.5]]), seed=1, dt=1e-3,
                                n_paths=4)
        m = r["mean"].cpu().numpy()
        assert np.isfinite(m[0]) and np.isnan(m[1]) and np.isnan(r["se"][1].item())
        # node_offset must keep the node stream indices within 32 bits
        with pytest.raises(PDDError):
            ctx.interface_solve(torch.tensor([[0.5, 0.5], [0.5, 0.4]]), seed=1, dt=1e-3,
                                n_paths=4, node_offset=2**32 - 1)
        # invalid arguments are rejected before any launch
        with pytest.raises(PDDError):
            ctx.interface_solve(torch.tensor([[0.5, 0.5]]), seed=1, dt=-1.0, n_paths=4)
        with pytest.raises(PDDError):
            ctx.interface_solve(torch.tensor([[0.5, 0.5]]), seed=1, dt=1e-3, n_paths=0)


def test_elliptic_full_size_closed_form(api):
    """The 4096-node, 1e5-path, dt = 1e-4 workload against the exact solution."""
    w = W.workload(2)
    with api.Context(w["prob"]) as ctx:
        r = ctx.interface_solve(torch.from_numpy(w["nodes"]), seed=w["seed"], dt=w["dt"],
                                n_paths=w["n_paths"], precision="fp32", diag=True)
    x = w["nodes"]
    exact = np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1]) * np.exp(x[:, 2])
    mean, se = r["mean"].cpu().numpy(), r["se"].cpu().numpy()
    z = (mean - exact) / se
    # Nodes within a few sqrt(dt) of the boundary carry the scheme's O(dt)
    # weak error of up to ~15 dt (measured with the FP64 oracle on the same
    # streams: it halves with dt), which there exceeds their small standard
    # error; the 4.5-sigma statistics apply beyond 5 sqrt(dt) from every face.
    dist = np.minimum(x, 1 - x).min(1)
    interior = dist > 5 * np.sqrt(w["dt"])
    print(f"full size: path-steps {r['path_steps']:.3e}, interior mean |z| "
          f"{np.abs(z[interior]).mean():.3f}, max |z| {np.abs(z[interior]).max():.2f}, "
          f"all-node max |err| {np.abs(mean - exact).max():.2e}, capped {r['capped']}")
    assert np.all(np.abs(mean - exact) <= 4.5 * se + 15 * w["dt"])
    zi = z[interior]
    assert np.all(np.abs(zi) <= 4.5)                  # 4096 nodes: 4.5 sigma
    assert abs(zi.mean()) < 0.25 and 0.8 < zi.std() < 1.25
    assert r["capped"] == 0


def test_elliptic_full_size_sampled_parity(api, orc):
    """Full-size launch (the benchmark's configuration); sampled nodes against
    the oracle path by path, on the full run's streams."""
    w = W.workload(2)
    sample = np.array([0, 1365, 2730, 4095])
    with api.Context(w["prob"]) as ctx:
        r = ctx.interface_solve(torch.from_numpy(w["nodes"]), seed=w["seed"], dt=w["dt"],
                                n_paths=w["n_paths"], precision="fp32", dump_paths=True)
        g = {"score": r["score"][sample], "steps": r["steps"][sample], "exit": r["exit"][sample]}
        mean_full = r["mean"][sample].clone()
        del r
        torch.cuda.empty_cache()
        # the same nodes solved on their own, keyed by their index in the
        # full list (node_offset), draw the same paths
        for j, i in enumerate(sample):
            one = ctx.interface_solve(torch.from_numpy(w["nodes"][i:i + 1]), seed=w["seed"],
                                      dt=w["dt"], n_paths=w["n_paths"], precision="fp32",
                                      node_offset=int(i))
            assert torch.equal(one["mean"][0], mean_full[j])
    o = orc.interface_solve(w["prob"], w["nodes"][sample], node_ids=sample, seed=w["seed"],
                            dt=w["dt"], n_paths=w["n_paths"], dump_paths=True)
    c = parity.compare_paths(g, o, prob=w["prob"], geometry="unit_cube")
    parity.check("elliptic3d fp32 full-size sampled", c, flip_max=FLIP_MAX_FP32)


def test_autotune_picks_a_shape_and_keeps_results(api):
    w = W.workload(2)
    nodes = torch.from_numpy(w["nodes"][::8])
    kw = dict(seed=w["seed"], dt=1e-3, n_paths=500, precision="fp32")
    with api.Context(w["prob"]) as ctx:
        before = ctx.interface_solve(nodes, **kw)["mean"].clone()
        t = ctx.autotune(nodes, repeats=1, **kw)
        after = ctx.interface_solve(nodes, **kw)["mean"]
    assert 1 <= t["blocks_per_sm"] <= 8 and t["ms"] > 0
    assert torch.equal(before, after)


@pytest.mark.parametrize("max_steps", [13, 30])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_step_cap_matches_oracle_path_by_path(api, orc, max_steps, precision):
    """Paths stopped by the step cap (a cap that falls inside a unit of four
    steps, after whole units) score g at the projection on the nearest face
    and report -max_steps, path by path as in the oracle."""
    w = W.workload(2)
    nodes = w["nodes"][::512]
    kw = dict(seed=w["seed"] + 7, dt=1e-5, n_paths=300, max_steps=max_steps)
    with api.Context(w["prob"]) as ctx:
        g = ctx.interface_solve(torch.from_numpy(nodes), precision=precision, dump_paths=True,
                                diag=True, **kw)
    o = orc.interface_solve(w["prob"], nodes, dump_paths=True, **kw)
    stg = g["steps"].cpu().numpy()
    assert (stg == -max_steps).mean() > 0.9            # most paths hit the cap
    assert g["capped"] == int((stg == -max_steps).sum())
    if precision == "fp64":
        c = parity.compare_paths(g, o, path_tol=1e-11, geometry="unit_cube")
    else:
        c = parity.compare_paths(g, o, prob=w["prob"], geometry="unit_cube")
    parity.check(f"elliptic3d step cap {max_steps} {precision}", c,
                 flip_max=1e-4 if precision == "fp64" else FLIP_MAX_FP32)


def test_batch_step_cap_matches_interface_solve(api):
    """The batch kernels' cap scoring (batch_capped) and the path kernel's
    (parked and scored with the exit queue) give the same paths."""
    w = W.workload(2)
    nodes = w["nodes"][::256]
    n, N, dt = len(nodes), 2000, 1e-5
    with api.Context(w["prob"]) as ctx:
        r = ctx.batch_solve([w["prob"]], torch.from_numpy(nodes), torch.zeros(n, dtype=torch.int32),
                            torch.full((n,), dt, dtype=torch.float64), seed=3, n_pilot=200,
                            n_min=N, n_max=N, target_se=1.0, max_steps=21, diag=True)
        p = ctx.interface_solve(torch.from_numpy(nodes), seed=3, dt=dt, n_paths=N,
                                precision="fp32", max_steps=21, diag=True)
    assert r["capped"] > 0 and r["capped"] == p["capped"]
    assert r["path_steps"] == p["path_steps"]
    np.testing.assert_allclose(r["mean"].cpu().numpy(), p["mean"].cpu().numpy(), rtol=1e-9,
                               atol=1e-12)
