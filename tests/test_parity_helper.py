"""CPU checks of the path-by-path parity helper (tests/parity.py) on planted
data: exit-step flips, exit-face flips and same-exit mismatches are told
apart and counted, and the node bar uses only same-exit paths."""
import numpy as np
import pytest

from tests import parity


def _fake(n=3, N=1000, dim=3, seed=0):
    rng = np.random.default_rng(seed)
    score = rng.normal(1.0, 0.5, (n, N))
    steps = rng.integers(1, 500, (n, N)).astype(np.int32)
    x = rng.uniform(0.1, 0.9, (n, N, dim))
    axis = rng.integers(0, dim, (n, N))
    side = rng.integers(0, 2, (n, N)).astype(np.float64)
    np.put_along_axis(x, axis[..., None], side[..., None], axis=2)
    return {"score": score, "steps": steps, "exit": x}


def test_exit_face_codes():
    x = np.array([[0.0, 0.3, 0.4], [0.2, 1.0, 0.4], [0.2, 0.3, 0.0], [0.0, 1.0, 0.5]])
    assert parity.exit_face(x, "unit_cube").tolist() == [0, 4, 6, 0]
    xl = np.array([[0.5, 0.7], [0.7, 0.5], [0.2, 0.0], [0.5, 0.5]])
    assert parity.exit_face(xl, "l_shape").tolist() == [2, 5, 3, 2]
    assert parity.exit_face(np.array([[0.5, 0.7]]), "unit_square").tolist() == [-1]


def test_planted_flips_and_mismatches_are_counted():
    o = _fake()
    g = {k: v.copy() for k, v in o.items()}
    g["score"] += 1e-7 * o["score"]                      # binary32-like noise
    g["steps"][0, 10] += 1                               # one exit-step flip
    g["score"][0, 10] += 0.3
    g["exit"][1, 20] = o["exit"][1, 20]                  # one exit-face flip at the same step
    ax = int(np.argmax((o["exit"][1, 20] == 0) | (o["exit"][1, 20] == 1)))
    g["exit"][1, 20, ax] = 0.5
    g["exit"][1, 20, (ax + 1) % 3] = 1.0 if o["exit"][1, 20, (ax + 1) % 3] != 1.0 else 0.0
    g["score"][1, 20] += 0.2
    st = parity.compare_paths(g, o, path_tol=1e-5, geometry="unit_cube")
    assert st["step_flips"] == 1 and st["face_flips"] == 1 and st["mismatch"] == 0
    assert st["flip_frac"] == pytest.approx(2 / 3000)
    assert st["node_rel_max"] < 1e-6
    parity.check("planted", st, flip_max=1e-3)
    g["score"][2, 5] += 1e-3                             # a same-exit path outside the bound
    st = parity.compare_paths(g, o, path_tol=1e-5, geometry="unit_cube")
    assert st["mismatch"] == 1
    with pytest.raises(AssertionError):
        parity.check("planted mismatch", st, flip_max=1e-3)


def test_without_exit_points_only_steps_classify():
    o = _fake(dim=2)
    g = {"score": o["score"].copy(), "steps": o["steps"].copy()}
    g["score"][0, 0] += 1.0
    st = parity.compare_paths(g, o, path_tol=1e-5)
    assert st["face_flips"] == 0 and st["mismatch"] == 1


def test_flip_limit_and_node_bar_enforced():
    o = _fake()
    g = {k: v.copy() for k, v in o.items()}
    g["steps"][:, :20] += 1
    st = parity.compare_paths(g, o, path_tol=1e-5, geometry="unit_cube")
    with pytest.raises(AssertionError):
        parity.check("too many flips", st, flip_max=1e-3)
    g = {k: v.copy() for k, v in o.items()}
    g["score"] = g["score"] * (1 + 5e-6)                 # within the path bound, biased
    st = parity.compare_paths(g, o, path_tol=1e-5, geometry="unit_cube")
    assert st["mismatch"] == 0
    with pytest.raises(AssertionError):
        parity.check("biased node", st, flip_max=1e-3, node_tol=1e-6)


@pytest.mark.parametrize("name", ["laplace", "elliptic", "fourier"])
def test_grad_norm_matches_finite_differences_of_g(orc, name):
    """|grad g| of the per-path bound against central differences of the
    oracle's boundary data g at random points."""
    from paper_1705_03666_gb300 import workloads as W
    prob = {"laplace": W.laplace_expcos(), "elliptic": W.elliptic_manufactured(),
            "fourier": W.workload(5)["prob"]}[name]
    d = int(prob["dim"])
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (20, d))
    h = 1e-6
    fd = np.zeros((20, d))
    for i in range(20):
        for k in range(d):
            xp, xm = x[i].copy(), x[i].copy()
            xp[k] += h
            xm[k] -= h
            fd[i, k] = (orc.eval_coeffs(prob, xp)[5] - orc.eval_coeffs(prob, xm)[5]) / (2 * h)
    np.testing.assert_allclose(parity.grad_norm(prob, x), np.linalg.norm(fd, axis=1),
                               rtol=1e-6, atol=1e-6)


def test_path_bound_grows_with_steps_and_gradient():
    from paper_1705_03666_gb300 import workloads as W
    prob = W.laplace_expcos()
    o = {"steps": np.array([[10, 1000, -30]]), "score": np.array([[1.0, 1.0, 1.0]]),
         "exit": np.array([[[0.0, 0.3], [0.0, 0.3], [1.0, 0.3]]])}
    b = parity.path_bound(prob, o)
    assert b[0, 1] > b[0, 0] and b[0, 2] > (38 / 18) * b[0, 0] * 0.9
    assert b[0, 0] == pytest.approx(2.0 ** -22 * (18 * 1.0 + 32))
