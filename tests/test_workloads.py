"""The seeded input recipes shared by the CUDA path and the oracle: each
generator reproduces the recipe it states (node placements, sizes, seeds),
deterministically, with every node where its problem needs it."""
import numpy as np

from paper_1705_03666_gb300 import workloads as W


def test_plastic_number_and_r2_sequence():
    p = W._PLASTIC
    assert abs(p ** 3 - p - 1.0) < 1e-14          # real root of x^3 = x + 1
    pts = W.r2_points(5)
    np.testing.assert_array_equal(pts[0], [0.5, 0.5])
    want = np.mod(0.5 + 3 * np.array([1 / p, 1 / p ** 2]), 1.0)
    np.testing.assert_allclose(pts[3], want, rtol=0, atol=1e-15)
    assert np.all((pts >= 0) & (pts < 1))


def test_laplace_nodes_on_the_interface():
    nodes = W.nodes_cfg1(16)
    assert nodes.shape == (16, 2)
    assert np.all(nodes[:, 0] == 0.5)
    np.testing.assert_array_equal(nodes[:, 1], np.arange(1, 17) / 17.0)


def test_cube_plane_rule():
    nodes = W.nodes_cube_planes(4096)
    assert nodes.shape == (4096, 3)
    pts = W.r2_points(4096 // 9 + 1)
    for n in (0, 1, 2, 3, 7, 8, 9, 100, 4095):
        a, j = n % 3, (n // 3) % 3
        assert nodes[n, a] == (j + 1) / 4.0
        others = [k for k in range(3) if k != a]
        np.testing.assert_array_equal(nodes[n, others], pts[n // 9])
    assert np.all((nodes > 0) & (nodes < 1))      # strictly inside the cube
    # nine planes, evenly used; a node repeats only where planes meet (R2
    # point 0 is (1/2, 1/2), so the three x_a = 1/2 nodes of the first group
    # are the centre): each node index still draws its own streams
    keys = [(n % 3, (n // 3) % 3) for n in range(4096)]
    counts = np.bincount([3 * a + j for a, j in keys], minlength=9)
    assert counts.min() >= 455 and counts.max() <= 456
    uniq, inv, cnt = np.unique(nodes, axis=0, return_inverse=True, return_counts=True)
    for u in uniq[cnt > 1]:
        assert np.all(np.isin(u, [0.25, 0.5, 0.75])), u
    assert len(uniq) >= 4090


def test_kpp_space_time_nodes():
    nodes = W.nodes_kpp()
    assert nodes.shape == (1024, 3)
    assert set(np.unique(nodes[:, 0])) == {-3.0, -1.0, 1.0, 3.0}
    np.testing.assert_allclose(np.unique(nodes[:, 1]), np.linspace(-2.0, 2.0, 16))
    np.testing.assert_allclose(np.unique(nodes[:, 2]), np.arange(1, 17) / 16.0)


def test_poisson_nodes_and_parameters():
    nodes = W.nodes_cfg5()
    assert nodes.shape == (2048, 2)
    assert set(np.unique(nodes[:, 0])) == {0.2, 0.4, 0.6, 0.8}
    np.testing.assert_array_equal(np.unique(nodes[:, 1]), np.arange(1, 513) / 513.0)
    prob = W.poisson_fourier()
    assert prob["params"].size == 80                  # 64 theta + 16 phi
    phi = prob["params"][64:]
    assert 0.02 < np.std(phi) < 0.3                    # phi ~ 0.1 N(0, 1)
    np.testing.assert_array_equal(W.poisson_fourier()["params"], prob["params"])


def test_lshape_interface_nodes_inside_the_l():
    nodes = W.nodes_lshape_interfaces(7001)
    assert nodes.shape == (7001, 2)
    on_x = nodes[:, 0] == 0.5
    on_y = nodes[:, 1] == 0.5
    assert np.all(on_x ^ on_y)
    assert np.all(nodes[on_x, 1] < 0.5) and np.all(nodes[on_y, 0] < 0.5)
    assert np.all((nodes > 0) & (nodes < 1))
    assert not np.any((nodes[:, 0] > 0.5) & (nodes[:, 1] > 0.5))   # not in the notch
    assert abs(int(on_x.sum()) - int(on_y.sum())) <= 1


def test_batch_mix_recipe():
    mix = W.batch_mix()
    n = 7000 + 7000 + 6000
    assert mix["nodes"].shape == (n, 3)
    np.testing.assert_array_equal(np.bincount(mix["problem_index"]), [7000, 7000, 6000])
    assert set(np.unique(mix["dt"])) == {1e-3, 1e-4}
    assert 0.45 < np.mean(mix["dt"] == 1e-3) < 0.55
    assert np.all(mix["nodes"][:14000, 2] == 0.0)     # 2-D families padded
    again = W.batch_mix()
    np.testing.assert_array_equal(again["dt"], mix["dt"])
    np.testing.assert_array_equal(again["nodes"], mix["nodes"])
    assert [p["geometry"] for p in mix["problems"]] == ["unit_square", "l_shape", "unit_cube"]


def test_workload_table():
    w1, w2, w4, w5 = (W.workload(k) for k in (1, 2, 4, 5))
    assert w1["nodes"].shape == (16, 2) and w1["n_paths"] == 10_000
    assert w1["dt"] == 1e-3 and w1["precision"] == "fp64"
    assert w2["nodes"].shape == (4096, 3) and w2["n_paths"] == 100_000
    assert w2["dt"] == 1e-4 and w2["precision"] == "fp32"
    assert w4["nodes"].shape == (1024, 3) and w4["n_trees"] == 100_000
    assert w5["nodes"].shape == (2048, 2) and w5["n_paths"] == 100_000
    for k, w in ((1, w1), (2, w2), (4, w4), (5, w5)):
        assert w["seed"] == W.SEED_BASE + k
    assert W.SEED_BASE == 0x1705036660000000
