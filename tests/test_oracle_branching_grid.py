"""Pins for the oracle's branching trees on a time grid (Algorithm 3.1: one
tree scores every T_i) with absorbing boundaries (Eq. 3.2).  Closed forms:
the spatially constant solution of the KPP ODE with matching boundary data,
the KPP travelling wave (exact on any domain when its trace is the boundary
data), the heat equation's first Dirichlet mode when branching is switched
off, and in free space the ODE of a general (marked) offspring law."""
import numpy as np
import pytest

from paper_1705_03666_gb300 import workloads as W

T8 = np.arange(1, 9) / 8.0


def _z(r, exact):
    return (r["mean"] - exact) / np.maximum(r["se"], 1e-300)


def test_constant_data_on_square_and_lshape(orc):
    """psi = c and g(x, s) = c / (c + (1 - c) e^{beta s}) give u(x, t) = that
    ODE solution everywhere (its Laplacian vanishes); checks the absorption
    time shift g(X_tau, t - tau)."""
    beta, c = 2.0, 0.3
    exact = c / (c + (1 - c) * np.exp(beta * T8))
    for geom, nodes in (("unit_square", np.array([[0.5, 0.5], [0.1, 0.7], [0.9, 0.05]])),
                        ("l_shape", np.array([[0.25, 0.75], [0.45, 0.45], [0.75, 0.25]]))):
        prob = W.kpp("const", c, beta, geometry=geom)
        r = orc.branching_grid_solve(prob, nodes, T8, seed=2, n_trees=20000, dt=2e-3)
        assert np.all(np.abs(_z(r, exact[None, :])) < 4.5), geom
        assert np.all(r["discarded"] == 0)


@pytest.mark.parametrize("beta", [1.0, 4.0])
def test_travelling_wave_on_square(orc, beta):
    a = np.sqrt(beta / 3.0)
    prob = W.kpp("travelling", a, beta, geometry="unit_square")
    nodes = np.array([[0.5, 0.5], [0.25, 0.3], [0.8, 0.6], [0.05, 0.5]])
    r = orc.branching_grid_solve(prob, nodes, T8, seed=3, n_trees=20000, dt=1e-3)
    exact = 1 - (1 + np.exp(a * nodes[:, :1] - 5 * beta * T8[None, :] / 6)) ** -2
    assert np.all(np.abs(r["mean"] - exact) < 4.5 * r["se"] + 2e-3)


def test_heat_mode_without_branching(orc):
    """beta -> 0: no particle ever branches and Eq. 3.2 is the heat equation
    with zero boundary data; psi = sin(pi x) sin(pi y) decays as
    exp(-pi^2 t) (1-D: exp(-pi^2 t / 2)).  O(dt) bias with the bridge."""
    for dim, geom, nodes in ((2, "unit_square", np.array([[0.5, 0.5], [0.3, 0.6]])),
                             (1, "interval", np.array([[0.5], [0.2]]))):
        prob = W.kpp("sine", 0.0, 1e-12, dim=dim, geometry=geom)
        T = np.array([0.02, 0.05, 0.1, 0.2])
        r = orc.branching_grid_solve(prob, nodes, T, seed=4, n_trees=40000, dt=1e-4)
        mode = np.prod(np.sin(np.pi * nodes), axis=1)[:, None]
        exact = mode * np.exp(-dim * np.pi ** 2 * T[None, :] / 2)
        assert np.all(np.abs(r["mean"] - exact) < 4.5 * r["se"] + 3e-3), (dim, _z(r, exact))


def test_bridge_reduces_absorption_bias(orc):
    """Without the bridge test the walk misses excursions out of the domain
    between steps (O(sqrt dt) bias); with it the bias is O(dt)."""
    prob = W.kpp("sine", 0.0, 1e-12, dim=1, geometry="interval")
    nodes = np.array([[0.5]])
    T = np.array([0.1])
    exact = np.exp(-np.pi ** 2 * 0.1 / 2)
    kw = dict(seed=5, n_trees=200000, dt=4e-3)
    e_off = orc.branching_grid_solve(prob, nodes, T, bridge=False, **kw)["mean"][0, 0] - exact
    e_on = orc.branching_grid_solve(prob, nodes, T, bridge=True, **kw)["mean"][0, 0] - exact
    assert e_off > 5 * abs(e_on) and e_off > 0.01


def test_free_space_marked_law_every_time_point(orc):
    """Free space, psi = c, offspring law q with marks alpha: u(t) solves
    v' = beta (sum_k alpha_k v^k - v) at every grid time from one tree per
    sample (weights enter only for branchings before each T_i)."""
    beta, c = 1.0, 0.4
    q = np.array([0.2, 0.3, 0.5])
    alpha = np.array([0.5, -0.2, 0.7])
    prob = W.kpp("const", c, beta, q=q, alpha=alpha, dim=1)
    T = np.array([0.25, 0.5, 0.75, 1.0])
    r = orc.branching_grid_solve(prob, np.array([[0.0], [3.0]]), T, seed=6, n_trees=100000)
    # RK4 on the ODE
    v, t, h, out = c, 0.0, 1e-4, []
    f = lambda v: beta * (alpha[0] + alpha[1] * v + alpha[2] * v * v - v)
    for Ti in T:
        while t < Ti - 1e-12:
            k1 = f(v); k2 = f(v + h / 2 * k1); k3 = f(v + h / 2 * k2); k4 = f(v + h * k3)
            v += h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
            t += h
        out.append(v)
    assert np.all(np.abs(_z(r, np.array(out)[None, :])) < 4.5)


def test_free_space_travelling_wave_and_ticks(orc):
    a = np.sqrt(1.0 / 3.0)
    prob = W.kpp("travelling", a, 1.0, dim=2)
    nodes = np.array([[-1.0, 0.0], [0.0, 2.0], [1.5, -1.0]])
    r = orc.branching_grid_solve(prob, nodes, T8, seed=7, n_trees=40000)
    exact = 1 - (1 + np.exp(a * nodes[:, :1] - 5 * T8[None, :] / 6)) ** -2
    assert np.all(np.abs(_z(r, exact)) < 4.5)
    assert orc.grid_ticks_per_unit(1.0) == 2.0 ** 30
    assert orc.grid_ticks_per_unit(0.75) == 2.0 ** 31
    assert orc.grid_ticks_per_unit(3.0) == 2.0 ** 29


def test_boundary_nodes_and_rejections(orc):
    prob = W.kpp("travelling", 0.5, 1.0, geometry="unit_square")
    r = orc.branching_grid_solve(prob, np.array([[0.0, 0.3]]), T8, seed=1, n_trees=10,
                                 dump_trees=True)
    exact = 1 - (1 + np.exp(-5 * T8 / 6)) ** -2
    assert np.allclose(r["score"][0], exact[None, :], rtol=1e-14) and np.all(r["steps"] == 0)
    with pytest.raises(ValueError):
        orc.branching_grid_solve(prob, np.array([[1.2, 0.3]]), T8, seed=1, n_trees=10)
    with pytest.raises(ValueError):
        orc.branching_grid_solve(prob, np.array([[0.5, 0.3]]), T8[::-1], seed=1, n_trees=10)
