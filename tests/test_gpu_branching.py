"""GPU parity of pdd_branching_solve against the FP64 oracle (shared streams).

Each tree consumes the same Philox words on both sides (depth-first particle
ids), so trees are compared one by one: a tree whose FP32 time bookkeeping
lands on the other side of t changes its segment count (a structure flip,
counted), and every other tree's score must agree within a per-tree bound
from the FP32 rounding of its positions and psi values (no exceptions).  Node means are
also pinned to the closed forms of Sec. 3.1-3.2 and, at full size, to a
Crank-Nicolson solution of the 1-D PDE (the data depend on x1 only).
"""
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


# Per-tree bound on the score difference of trees with the same structure,
# in units of 2^-22 (segments + 4) max(1, |s|): every segment rounds the
# particle's binary32 position and evaluates psi with the hardware exp2 and
# reciprocal (a few ulp), and the float-float product adds ~2^-44 per factor.
# Measured on GB300: at most 1.08 of the unit.
TREE_FACTOR = 4.0


def _tree_compare(g, o, name):
    """Tree by tree: a different segment count, or a tree pruned on one side
    only, is a structure flip (counted); every other tree must agree within
    the per-tree bound (none may exceed it).  Node means over the unflipped
    trees, relative difference."""
    sg, so = g["score"].cpu().numpy(), o["score"]
    gg, go = g["segs"].cpu().numpy(), o["segments"]
    nan_g, nan_o = np.isnan(sg), np.isnan(so)
    same = (gg == go) & (nan_g == nan_o)
    unit = 2.0 ** -22 * (np.abs(go) + 4.0) * np.maximum(1.0, np.abs(so))
    ratio = np.where(same & ~nan_o, np.abs(sg - so) / unit, 0.0)
    mismatch = int((ratio > TREE_FACTOR).sum())
    m = same & ~nan_o
    cnt = m.sum(1)
    mg = np.where(m, sg, 0).sum(1) / np.maximum(cnt, 1)
    mo = np.where(m, so, 0).sum(1) / np.maximum(cnt, 1)
    rel = np.abs(mg - mo) / np.maximum(np.abs(mo), 1e-3)
    flips = 1.0 - same.mean()
    print(f"[parity] {name}: tree flips {flips:.2e} ({int((~same).sum())} of {same.size}), "
          f"mismatches {mismatch}, max ratio to 2^-22 (segs + 4) {ratio.max():.3f}, "
          f"max node rel {rel.max():.2e}")
    assert mismatch == 0, (name, ratio.max())
    return flips, rel


@pytest.mark.parametrize("prob_args,dim", [
    (dict(psi="sigmoid", psi_param=4.0), 2),
    (dict(psi="travelling", psi_param=1 / np.sqrt(3.0)), 1),
    (dict(psi="const", psi_param=0.4, q=(0.5, 0.0, 0.5)), 1),
    (dict(psi="const", psi_param=0.6, q=(0.25, 0.25, 0.25, 0.0, 0.25),
          alpha=(0.0586, 0.5, 0.8199, 0.0, -0.4095)), 1),
])
def test_trees_match_oracle(api, orc, prob_args, dim):
    prob = W.kpp(dim=dim, **prob_args)
    nodes = W.nodes_kpp(n_x2=4, n_t=8)[::3]
    if dim == 1:
        nodes = nodes[:, [0, 2]]
    kw = dict(seed=W.SEED_BASE + 4, n_trees=3001, max_particles=4096, max_depth=64)
    with api.Context(prob) as ctx:
        g = ctx.branching_solve(torch.from_numpy(nodes), dump_trees=True, **kw)
    o = orc.branching_solve(prob, nodes, dump_trees=True, **kw)
    flips, rel = _tree_compare(g, o, f"trees {prob_args['psi']} d={dim}")
    assert flips <= 1e-4
    assert rel.max() <= 1e-5
    assert g["segments"] == int(np.abs(o["segments"]).sum())


def test_caps_match_oracle(api, orc):
    prob = W.kpp("const", 0.5, 1.0, dim=1)
    nodes = np.array([[0.0, 2.0], [1.0, 1.5]])
    kw = dict(seed=7, n_trees=5000, max_particles=6, max_depth=3)
    with api.Context(prob) as ctx:
        g = ctx.branching_solve(torch.from_numpy(nodes), dump_trees=True, **kw)
    o = orc.branching_solve(prob, nodes, dump_trees=True, **kw)
    assert g["status"] == 5 and g["discarded"] == int(o["discarded"].sum()) > 0
    assert np.array_equal(g["n"].cpu().numpy(), o["n"])
    assert np.array_equal(np.isnan(g["score"].cpu().numpy()), np.isnan(o["score"]))


def test_kpp_constant_data_closed_form(api):
    prob = W.kpp("const", 0.3, 1.0, dim=2)
    ts = np.linspace(0.1, 1.0, 10)
    nodes = np.stack([np.zeros_like(ts), np.zeros_like(ts), ts], 1)
    with api.Context(prob) as ctx:
        r = ctx.branching_solve(torch.from_numpy(nodes), seed=3, n_trees=200000)
    exact = 0.3 / (0.3 + 0.7 * np.exp(ts))
    m, se = r["mean"].cpu().numpy(), r["se"].cpu().numpy()
    assert np.all(np.abs(m - exact) <= 3.5 * se)


def test_kpp_workload_full_size(api):
    """The 1024-node, 1e5-tree workload: u depends on x1 and t only; compare
    against Crank-Nicolson of the 1-D PDE."""
    from test_oracle_branching import _cn_kpp_sigmoid
    w = W.workload(4)
    with api.Context(w["prob"]) as ctx:
        r = ctx.branching_solve(torch.from_numpy(w["nodes"]), seed=w["seed"],
                                n_trees=w["n_trees"], max_particles=w["max_particles"],
                                max_depth=w["max_depth"], diag=True)
    m, se = r["mean"].cpu().numpy(), r["se"].cpu().numpy()
    x1, t = w["nodes"][:, 0], w["nodes"][:, 2]
    ref = np.zeros_like(m)
    for tt in np.unique(t):
        xg, ug = _cn_kpp_sigmoid(4.0, float(tt), dx=4e-3, dt=float(tt) / 400)
        sel = t == tt
        ref[sel] = np.interp(x1[sel], xg, ug)
    z = (m - ref) / se
    print(f"kpp full: segments {r['segments']:.3e}, mean z {z.mean():.3f}, std z {z.std():.3f}")
    assert r["discarded"] == 0
    assert np.all(np.abs(m - ref) <= 4.5 * se + 5e-4)
    assert abs(z.mean()) < 0.3


def test_large_trees_match_oracle(api, orc):
    """beta = 6 at t = 1: ~600 segments per tree on average and trees of
    thousands (pruned above 4096), the regime where a binary32 product of the
    leaves' psi values would drift; the tree products are accumulated as
    float-float values and compared tree by tree with the FP64 oracle.

    Per-tree bound (first-order error model of the binary32 positions): every
    segment moves its particle with one or two binary32 roundings (2^-23
    relative to |x| + 1) and every leaf's psi carries those of its lineage
    times |psi'/psi| <= a (the sigmoid's steepness, 4) plus a few ulp of its
    own evaluation, so a tree of n segments satisfies
        |s_gpu - s_oracle| <= 2^-20 (n + 8) a (1 + max|x|) |s|.
    Measured on GB300 the largest relative difference is 8e-5 (trees of
    ~600 segments; the bound there is ~2e-2): per-tree agreement at 1e-5 is
    out of reach of binary32 positions for trees this size, which is why the
    node means over the trees of equal structure carry the 1e-5 bar."""
    prob = W.kpp("sigmoid", 4.0, beta=6.0, dim=2)
    nodes = np.array([[-1.0, 0.0, 1.0], [0.0, 0.5, 1.0], [1.0, -0.5, 1.0], [0.5, 0.0, 0.6]])
    kw = dict(seed=W.SEED_BASE + 44, n_trees=4000, max_particles=4096, max_depth=64)
    with api.Context(prob) as ctx:
        g = ctx.branching_solve(torch.from_numpy(nodes), dump_trees=True, diag=True, **kw)
    o = orc.branching_solve(prob, nodes, dump_trees=True, **kw)
    sg, so = g["score"].cpu().numpy(), o["score"]
    gg, go = g["segs"].cpu().numpy(), o["segments"]
    same = (gg == go) & ~np.isnan(so) & ~np.isnan(sg)
    rel = np.where(same, np.abs(sg - so) / np.maximum(np.abs(so), 1e-30), 0.0)
    bound = 2.0 ** -20 * (np.abs(go) + 8) * 4.0 * (1 + 8.0)
    print(f"large trees: {same.sum()} same-structure trees of {so.size}, max segments "
          f"{np.abs(go).max()}, mean {np.abs(go).mean():.0f}, structure flips "
          f"{(gg != go).sum()}, discarded {int(np.isnan(so).sum())}; per-tree rel max "
          f"{rel.max():.2e} ({(rel / bound).max():.3f} of the bound), 99.9% "
          f"{np.quantile(rel[same], 0.999):.2e}")
    assert np.all(rel <= bound)
    assert (gg != go).mean() <= 1e-3
    assert np.array_equal(np.isnan(sg), np.isnan(so))
    assert g["discarded"] == int(np.isnan(so).sum()) > 0
    flags = g["flags"].cpu().numpy()
    assert np.array_equal(flags & 8 != 0, np.isnan(so).any(1))   # PDD_NODE_DISCARDED
    mg = np.where(same, sg, 0).sum(1) / same.sum(1)
    mo = np.where(same, so, 0).sum(1) / same.sum(1)
    assert np.max(np.abs(mg - mo) / np.maximum(np.abs(mo), 1e-3)) <= 1e-5
