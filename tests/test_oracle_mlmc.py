"""Pins for the oracle's multilevel estimator (Sec. 2.1 names Giles'
multilevel method for the Euler scheme): the telescoping sum reproduces the
harmonic solution; each coupled coarse path has the law of the previous
level's fine path (so a wrong coarse step size fails); level 0 is the plain
scheme; and the level variances of P_l - P_{l-1} decay (about R^-1/2 per
level for exit problems, against a constant variance of P_l itself)."""
import numpy as np

from paper_1705_03666_gb300 import workloads as W


def test_mlmc_matches_harmonic(orc):
    prob = W.laplace_expcos()
    nodes = W.nodes_cfg1(4)
    r = orc.mlmc_solve(prob, nodes, seed=2, dt0=4e-3, n_per_level=[40000, 20000, 10000, 5000])
    exact = np.exp(nodes[:, 0]) * np.cos(nodes[:, 1])
    # bias of the finest level (dt = 5e-4, bridge on) is O(dt)
    assert np.all(np.abs(r["mean"] - exact) < 4.5 * r["se"] + 2e-3)


def test_coarse_paths_have_the_previous_levels_law(orc):
    """1-D torsion (u = x(1 - x)) with a coarse dt0 = 0.02 and the plain exit
    test, so every level is visibly biased: the coarse mean of level l must
    match the fine mean of level l-1 and differ from the fine mean of l."""
    prob = W.torsion("interval", 1)
    nodes = np.array([[0.3], [0.5]])
    kw = dict(seed=7, dt0=0.02, refine=2, n_paths=200000, bridge=False)
    L = [orc.mlmc_level(prob, nodes, level=l, **kw) for l in range(3)]
    se = np.sqrt(0.25 / 200000) * 2           # generous SE of a mean of E[tau]-like scores
    for l in (1, 2):
        assert np.all(np.abs(L[l]["coarse_mean"] - L[l - 1]["fine_mean"]) < 4.5 * se)
    exact = nodes[:, 0] * (1 - nodes[:, 0])
    bias0 = L[0]["fine_mean"] - exact
    assert np.all(np.abs(bias0) > 10 * se)      # the plain scheme is biased at dt0
    assert np.all(np.abs(L[1]["fine_mean"] - L[1]["coarse_mean"]) > 3 * se)


def test_level_zero_is_the_plain_scheme(orc):
    prob = W.laplace_expcos()
    nodes = W.nodes_cfg1(3)
    a = orc.mlmc_level(prob, nodes, seed=3, dt0=2e-3, level=0, n_paths=40000)
    b = orc.interface_solve(prob, nodes, seed=4, dt=2e-3, n_paths=40000)
    comb = np.sqrt(a["var"] / 40000 + b["se"] ** 2)
    assert np.all(np.abs(a["mean"] - b["mean"]) < 4.5 * comb)
    assert np.all(a["coarse_mean"] == 0)


def test_level_variances_decay(orc):
    prob = W.laplace_expcos()
    nodes = np.array([[0.5, 0.5], [0.5, 0.2]])
    V = [orc.mlmc_level(prob, nodes, seed=5, dt0=4e-3, level=l, n_paths=20000)["var"]
         for l in range(5)]
    assert np.all(V[1] < 0.2 * V[0])
    for l in range(1, 4):
        assert np.all(V[l + 1] < 0.95 * V[l]), (l, V[l], V[l + 1])
    # the finest pair of levels decays at least like R^-1/4 per level on average
    assert np.all(V[4] < V[1] * 0.5 ** 0.75)


def test_dumped_walk_records(orc):
    """The per-pair records: the pair's difference is the fine score minus
    the coarse score; each walk's exit point lies on the boundary with its
    score g there (e^x cos y; no source or killing in this family); the fine
    walk's exit step is the pair's step count or less, and the coarse exit
    step times the refinement is within one coarse step of it."""
    prob = W.laplace_expcos()
    nodes = np.array([[0.3, 0.4], [0.6, 0.7]])
    r = orc.mlmc_level(prob, nodes, seed=5, dt0=4e-3, level=2, refine=2, n_paths=400,
                       dump_paths=True)
    a = r["aux"]
    np.testing.assert_array_equal(r["diff"], a[..., 0] - a[..., 1])
    for which in (0, 1):
        x = a[..., 4 + 2 * which:6 + 2 * which]
        on = (x == 0.0) | (x == 1.0)
        assert on.any(-1).all()
        np.testing.assert_allclose(a[..., which], np.exp(x[..., 0]) * np.cos(x[..., 1]),
                                   rtol=1e-13)
    kf, kc = a[..., 2], a[..., 3]
    assert np.all((kf > 0) & (kf <= r["steps"]) & (kc > 0))
    assert np.all(np.maximum(kf, 2 * kc) == r["steps"])
