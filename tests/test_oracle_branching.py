"""Pins for the oracle's branching-diffusion estimator (CPU only).

Sec. 3.1 (Eq. 3.1, Assumption 3.1) and Sec. 3.2 (marked weights alpha/q):
  - constant initial data reduce the PDE to the ODE u' = beta (F(u) - u), whose
    solutions are closed forms for KPP (F = u^2) and for the die-or-split example
    of Sec. 3.1 (F = (1 + u^2)/2), and an RK4 integration for the marked
    polynomial F of Sec. 3.2 (negative coefficient, so weights alpha/q matter);
  - the KPP travelling wave printed in Sec. 3.1.1, rescaled to the (1/2) Lap
    generator used here;
  - the sigmoid initial data of the KPP workload against a Crank-Nicolson
    solve of the 1-D PDE, and independence of x2 in 2-D.
"""
import math

import numpy as np
import pytest

from paper_1705_03666_gb300 import workloads as W


def _within(mean, se, exact, bias=0.0):
    return np.all(np.abs(mean - exact) <= 3.0 * se + bias)


def test_kpp_constant_data_closed_form(orc):
    """psi = c: u = c / (c + (1 - c) e^{beta t})."""
    for beta, c in ((1.0, 0.3), (2.0, 0.7)):
        prob = W.kpp("const", c, beta, dim=1)
        ts = np.array([0.25, 0.5, 1.0])
        nodes = np.stack([np.zeros_like(ts), ts], axis=1)
        r = orc.branching_solve(prob, nodes, seed=1, n_trees=20000)
        exact = c / (c + (1 - c) * np.exp(beta * ts))
        assert _within(r["mean"], r["se"], exact)
        assert np.all(r["discarded"] == 0)


def test_die_or_split_closed_form(orc):
    """Sec. 3.1 example: alpha_0 = alpha_2 = 1/2, beta = 1.  Constant data c:
    u' = (1 - u)^2 / 2, so 1/(1 - u) = 1/(1 - c) + t/2."""
    c = 0.4
    prob = W.kpp("const", c, 1.0, q=(0.5, 0.0, 0.5), dim=1)
    ts = np.array([0.5, 1.0, 2.0])
    nodes = np.stack([np.zeros_like(ts), ts], axis=1)
    r = orc.branching_solve(prob, nodes, seed=2, n_trees=20000)
    exact = 1.0 - 1.0 / (1.0 / (1.0 - c) + ts / 2.0)
    assert _within(r["mean"], r["se"], exact)


def _rk4(F, u0, beta, t, n=4000):
    u, h = u0, t / n
    f = lambda v: beta * (F(v) - v)
    for _ in range(n):
        k1 = f(u); k2 = f(u + h * k1 / 2); k3 = f(u + h * k2 / 2); k4 = f(u + h * k3)
        u += h * (k1 + 2 * k2 + 2 * k3 + k4) / 6
    return u


def test_marked_polynomial_constant_data(orc):
    """Sec. 3.2: F(v) = 0.0586 + 0.5 v + 0.8199 v^2 - 0.4095 v^4 (the quartic of
    the CVA example), negative alpha_4, sampled with q = (1/4, 1/4, 1/4, 0, 1/4)
    and weights alpha/q.  Constant data: ODE v' = beta (F(v) - v)."""
    alpha = (0.0586, 0.5, 0.8199, 0.0, -0.4095)
    q = (0.25, 0.25, 0.25, 0.0, 0.25)
    F = lambda v: alpha[0] + alpha[1] * v + alpha[2] * v ** 2 + alpha[4] * v ** 4
    for c in (0.6, -0.5):
        prob = W.kpp("const", c, 1.0, q=q, alpha=alpha, dim=1)
        ts = np.array([0.3, 0.6])
        nodes = np.stack([np.zeros_like(ts), ts], axis=1)
        r = orc.branching_solve(prob, nodes, seed=3, n_trees=40000)
        exact = np.array([_rk4(F, c, 1.0, t) for t in ts])
        assert _within(r["mean"], r["se"], exact)


def test_marked_weights_matter(orc):
    """Sampling the marked problem with q but ignoring the weights (alpha = q)
    gives a different answer, which the ODE pin rejects."""
    alpha = (0.0586, 0.5, 0.8199, 0.0, -0.4095)
    q = (0.25, 0.25, 0.25, 0.0, 0.25)
    F = lambda v: alpha[0] + alpha[1] * v + alpha[2] * v ** 2 + alpha[4] * v ** 4
    prob = W.kpp("const", 0.6, 1.0, q=q, alpha=q, dim=1)
    nodes = np.array([[0.0, 0.6]])
    r = orc.branching_solve(prob, nodes, seed=3, n_trees=40000)
    assert not _within(r["mean"], r["se"], np.array([_rk4(F, 0.6, 1.0, 0.6)]))


def test_travelling_wave(orc):
    """Sec. 3.1.1 exact KPP wave, rescaled from u_xx to (1/2) u_xx:
    psi(x) = 1 - (1 + e^{x/sqrt3})^-2, u = 1 - (1 + e^{x/sqrt3 - 5t/6})^-2."""
    a = 1.0 / math.sqrt(3.0)
    prob = W.kpp("travelling", a, 1.0, dim=1)
    xs = np.array([-2.0, 0.0, 1.5, 3.0])
    ts = np.array([0.5, 1.0, 0.75, 0.25])
    r = orc.branching_solve(prob, np.stack([xs, ts], 1), seed=4, n_trees=20000)
    exact = 1.0 - (1.0 + np.exp(a * xs - 5.0 * ts / 6.0)) ** -2
    assert _within(r["mean"], r["se"], exact)


def _cn_kpp_sigmoid(slope, t_end, L=12.0, dx=4e-3, dt=1e-3):
    """Crank-Nicolson for u_t = (1/2) u_xx + u^2 - u on [-L, L] with the
    reaction term by Heun's method (Strang splitting), Dirichlet 0 and 1."""
    from scipy.linalg import solve_banded
    x = np.arange(-L, L + dx / 2, dx)
    u = 1.0 / (1.0 + np.exp(-slope * x))
    n = x.size - 2
    r = 0.5 * dt / dx ** 2
    ab = np.zeros((3, n))
    ab[0, 1:] = -r / 2
    ab[1] = 1 + r
    ab[2, :-1] = -r / 2
    steps = int(round(t_end / dt))
    react = lambda v: v * v - v
    for _ in range(steps):
        h = dt / 2
        u = u + h * (react(u) + react(u + h * react(u))) / 2
        rhs = u[1:-1] * (1 - r) + (r / 2) * (u[2:] + u[:-2])
        rhs[0] += (r / 2) * u[0] * 2
        rhs[-1] += (r / 2) * u[-1] * 2
        u[1:-1] = solve_banded((1, 1), ab, rhs)
        u = u + h * (react(u) + react(u + h * react(u))) / 2
        u[0], u[-1] = 0.0, 1.0
    return x, u


def test_kpp_sigmoid_vs_crank_nicolson(orc):
    """The KPP workload's initial data psi = 1/(1 + e^{-4 x1}) in 1-D."""
    xg, ug = _cn_kpp_sigmoid(4.0, 1.0)
    xg2, ug2 = _cn_kpp_sigmoid(4.0, 1.0, dx=2e-3, dt=5e-4)
    xs = np.array([-1.0, 0.0, 0.5, 2.0])
    e1, e2 = np.interp(xs, xg, ug), np.interp(xs, xg2, ug2)
    assert np.max(np.abs(e1 - e2)) < 2e-4  # the reference itself is converged
    prob = W.kpp("sigmoid", 4.0, 1.0, dim=1)
    r = orc.branching_solve(prob, np.stack([xs, np.ones_like(xs)], 1), seed=5,
                            n_trees=20000)
    assert _within(r["mean"], r["se"], e2, 3e-4)


def test_kpp_2d_independent_of_x2(orc):
    """psi depends on x1 only, so u(x1, x2, t) does not depend on x2; the 2-D
    estimate at the workload's nodes matches the 1-D CN solution."""
    xg, ug = _cn_kpp_sigmoid(4.0, 1.0, dx=2e-3, dt=5e-4)
    nodes = np.array([[-1.0, -2.0, 1.0], [-1.0, 2.0, 1.0], [1.0, 0.0, 1.0]])
    r = orc.branching_solve(W.kpp("sigmoid", 4.0, 1.0), nodes, seed=6,
                            n_trees=20000)
    assert _within(r["mean"], r["se"], np.interp(nodes[:, 0], xg, ug), 3e-4)


def test_tree_cap_discards_and_counts(orc):
    prob = W.kpp("const", 0.5, 1.0, dim=1)
    nodes = np.array([[0.0, 2.0]])
    r = orc.branching_solve(prob, nodes, seed=7, n_trees=2000, max_particles=3,
                            dump_trees=True)
    disc = r["discarded"][0]
    assert disc > 0 and r["n"][0] + disc == 2000
    assert np.isnan(r["score"][0]).sum() == disc
    assert np.all(r["segments"][0][np.isnan(r["score"][0])] < 0)
    # P(no branching before t=2) = e^{-2}: trees with one particle all kept
    assert np.all(r["segments"][0] != 0)


def test_segments_mean(orc):
    """Binary branching at rate beta: E[#segments] = 2 e^{beta t} - 1."""
    prob = W.kpp("const", 0.5, 1.0, dim=1)
    nodes = np.array([[0.0, 1.0]])
    r = orc.branching_solve(prob, nodes, seed=8, n_trees=40000, dump_trees=True)
    seg = r["segments"][0].astype(np.float64)
    assert abs(seg.mean() - (2 * math.e - 1)) < 4 * seg.std() / math.sqrt(seg.size)
