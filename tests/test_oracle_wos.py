"""Pins for the oracle's Walk on Spheres (Sec. 2.1; Eq. 1.1): harmonic data
are reproduced (mean-value property) on the square and the L-shape, the bias
is O(eps), non-harmonic data are not reproduced (sensitivity), boundary nodes
exit at once, and the walk needs O(log 1/eps) jumps."""
import numpy as np

from paper_1705_03666_gb300 import workloads as W


def test_harmonic_square_and_lshape(orc):
    for geom, pts in (("unit_square", W.nodes_cfg1(16)),
                      ("l_shape", np.array([[0.25, 0.75], [0.75, 0.25], [0.4, 0.4], [0.1, 0.5]]))):
        r = orc.wos_solve(W.laplace_expcos(geom), pts, seed=3, n_paths=40000, eps=1e-5)
        exact = np.exp(pts[:, 0]) * np.cos(pts[:, 1])
        assert np.all(np.abs(r["mean"] - exact) <= 4 * r["se"] + 1e-4), geom  # 20 nodes


def test_bias_is_order_eps(orc):
    """With a coarse shell the estimate is biased by O(eps) (the walk stops up
    to eps from the boundary and scores the projection); the bias shrinks
    with eps."""
    pts = np.array([[0.5, 0.3], [0.5, 0.7]])
    exact = np.exp(pts[:, 0]) * np.cos(pts[:, 1])
    errs = []
    for eps in (0.2, 0.05):
        r = orc.wos_solve(W.laplace_expcos(), pts, seed=5, n_paths=200000, eps=eps)
        errs.append(np.abs(r["mean"] - exact).max())
    assert errs[0] > 3 * errs[1] and errs[0] < 0.2


def test_jumps_grow_like_log_eps(orc):
    pts = np.array([[0.5, 0.5]])
    s = []
    for eps in (1e-2, 1e-4, 1e-6):
        r = orc.wos_solve(W.laplace_expcos(), pts, seed=1, n_paths=20000, eps=eps)
        s.append(r["total_steps"] / 20000)
    # each decade of eps adds a constant number of jumps
    d1, d2 = s[1] - s[0], s[2] - s[1]
    assert d1 > 1 and abs(d1 - d2) < 0.3 * d1


def test_boundary_node_and_streams(orc):
    nodes = np.array([[0.0, 0.4], [0.5, 0.5]])
    r = orc.wos_solve(W.laplace_expcos(), nodes, seed=1, n_paths=50, eps=1e-4, dump_paths=True)
    assert np.all(r["steps"][0] == 0) and np.all(r["score"][0] == np.cos(0.4))
    sub = orc.wos_solve(W.laplace_expcos(), nodes[1:], node_ids=[1], seed=1, n_paths=50,
                        eps=1e-4, dump_paths=True)
    assert np.array_equal(sub["score"][0], r["score"][1])


def test_dumped_stopping_points(orc):
    """The per-walk records: each stopping point lies on the boundary (a
    coordinate exactly on a face plane: 0, 1, or 1/2 on the L-shape's notch)
    and the walk's score is g there, e^x cos y."""
    for geom in ("unit_square", "l_shape"):
        prob = W.laplace_expcos(geom)
        nodes = np.array([[0.3, 0.4], [0.45, 0.2]])
        r = orc.wos_solve(prob, nodes, seed=3, n_paths=300, eps=1e-3, dump_paths=True)
        x = r["exit"]
        planes = (0.0, 1.0, 0.5) if geom == "l_shape" else (0.0, 1.0)
        on = np.zeros(x.shape[:2], dtype=bool)
        for v in planes:
            on |= (x[..., 0] == v) | (x[..., 1] == v)
        assert on.all()
        np.testing.assert_allclose(r["score"], np.exp(x[..., 0]) * np.cos(x[..., 1]), rtol=1e-15)
