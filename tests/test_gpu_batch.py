"""GPU checks of pdd_batch_solve (heterogeneous, variance-adaptive, one
persistent launch per pass, optionally captured in a CUDA graph).

The batch runs node i's paths on the streams pdd_interface_solve uses, with
the same step arithmetic and the same exact per-node sums, so a non-adaptive
batch (n_min = n_max = N) must reproduce pdd_interface_solve's node means and
standard errors bit for bit.
The adaptive path counts must follow the pilot variances, and the L-shape
(which only the batch and the plain solve support) is checked against the
oracle path by path.
"""
import numpy as np
import pytest
import torch

from paper_1705_03666_gb300 import workloads as W
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1705_03666_gb300 import api as a
    return a


def _small_mix():
    mix = W.batch_mix(square=40, lshape=40, cube=48, seed=11)
    return mix


def _reference_by_group(api, mix, seed, n_paths):
    """pdd_interface_solve per (problem, dt) group on the batch's node indices."""
    ref_m = np.zeros(len(mix["nodes"]))
    ref_s = np.zeros(len(mix["nodes"]))
    for p, prob in enumerate(mix["problems"]):
        for dt in (1e-3, 1e-4):
            sel = np.where((mix["problem_index"] == p) & (mix["dt"] == dt))[0]
            if len(sel) == 0:
                continue
            # place the group's nodes at their batch indices; other rows sit on
            # the boundary (zero cost, never read)
            dim = prob["dim"]
            full = np.zeros((sel.max() + 1, dim))
            full[:, 0] = 0.0
            full[:, 1:] = 0.25
            full[sel] = mix["nodes"][sel, :dim]
            with api.Context(prob) as ctx:
                r = ctx.interface_solve(torch.from_numpy(full), seed=seed, dt=dt, n_paths=n_paths,
                                        precision="fp32")
            ref_m[sel] = r["mean"].cpu().numpy()[sel]
            ref_s[sel] = r["se"].cpu().numpy()[sel]
    return ref_m, ref_s


@pytest.mark.parametrize("use_graph", [False, True])
def test_fixed_count_batch_equals_interface_solve(api, use_graph):
    mix = _small_mix()
    seed, N = 99, 1500
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with api.Context(mix["problems"][0]) as ctx:
            kw = dict(seed=seed, n_pilot=300, n_min=N, n_max=N, target_se=1.0, chunk=128,
                      use_graph=use_graph)
            r1 = ctx.batch_solve(mix["problems"], torch.from_numpy(mix["nodes"]),
                                 torch.from_numpy(mix["problem_index"]),
                                 torch.from_numpy(mix["dt"]), **kw)
            m1 = r1["mean"].cpu().numpy().copy()
            r2 = ctx.batch_solve(mix["problems"], torch.from_numpy(mix["nodes"]),
                                 torch.from_numpy(mix["problem_index"]),
                                 torch.from_numpy(mix["dt"]), **kw)   # replay
            m2 = r2["mean"].cpu().numpy()
        stream.synchronize()
    assert np.array_equal(m1, m2)
    assert np.all(r1["n"].cpu().numpy() == N)
    ref_m, ref_s = _reference_by_group(api, mix, seed, N)
    # both add each node's scores to exact integer sums: the same bits
    np.testing.assert_array_equal(m1, ref_m)
    np.testing.assert_array_equal(r1["se"].cpu().numpy(), ref_s)


def test_adaptive_counts_follow_pilot_variance(api):
    mix = _small_mix()
    seed, n_pilot, se_t = 5, 400, 3e-3
    with api.Context(mix["problems"][0]) as ctx:
        r = ctx.batch_solve(mix["problems"], torch.from_numpy(mix["nodes"]),
                            torch.from_numpy(mix["problem_index"]), torch.from_numpy(mix["dt"]),
                            seed=seed, n_pilot=n_pilot, n_min=500, n_max=20000, target_se=se_t,
                            diag=True)
    Ni = r["n"].cpu().numpy()
    # pilot statistics from the plain solve on the same streams
    pm, ps = _reference_by_group(api, mix, seed, n_pilot)
    var = ps ** 2 * n_pilot
    expect = np.clip(np.ceil(var / se_t ** 2), 500, 20000)
    assert np.all(np.abs(Ni - expect) <= 1)
    se = r["se"].cpu().numpy()
    ok = (Ni < 20000) & (Ni > 500)
    # where N_i is set by the pilot: SE_final = sqrt(var_final / N_i) and
    # N_i ~ var_pilot / SE*^2, so SE_final / SE* ~ sqrt(var_final / var_pilot)
    var_final = se ** 2 * Ni
    ratio = se[ok] / (se_t * np.sqrt(var_final[ok] / var[ok]))
    assert np.all(np.abs(ratio - 1.0) < 0.02)
    assert 0.85 < np.median(se[ok] / se_t) < 1.15   # the pilot is unbiased for var
    assert r["capped"] == 0 and r["path_steps"] > 0
    # per-node flags: the target not reached exactly where se > target_se
    flags = r["flags"].cpu().numpy()
    assert np.array_equal((flags & 32) != 0, se > se_t) and np.any(se > se_t)


def test_lshape_matches_oracle(api, orc):
    prob = W.laplace_expcos("l_shape")
    nodes = W.nodes_lshape_interfaces(24)
    kw = dict(seed=17, dt=1e-3, n_paths=2000)
    with api.Context(prob) as ctx:
        g = ctx.interface_solve(torch.from_numpy(nodes), precision="fp32", dump_paths=True, **kw)
    o = orc.interface_solve(prob, nodes, dump_paths=True, **kw)
    c = parity.compare_paths(g, o, prob=prob, geometry="l_shape")
    parity.check("l_shape fp32", c, flip_max=2e-4)
    exact = np.exp(nodes[:, 0]) * np.cos(nodes[:, 1])
    m, se = g["mean"].cpu().numpy(), g["se"].cpu().numpy()
    assert np.all(np.abs(m - exact) <= 4 * se + 5e-3)
