"""Pins for the oracle's diffusion-path estimator (CPU only).

The oracle follows the Feynman-Kac / Dynkin representation (Eq. 2.1-2.2 and
Eq. 2.5-2.9 in the elliptic Dirichlet reduction of Sec. 2.2) with
Euler-Maruyama steps and the boundary-corrected exit test cited in Sec. 2.1.
It is pinned to things that do not come from the oracle itself: closed-form
PDE solutions, a brute-force finite-difference solve, a symbolic derivation of
a manufactured source, a series solution, the convergence rates stated in
Sec. 2.1 and exact invariants.  A dropped term (drift, killing, source), a
wrong sign, a transposed coordinate or a broken exit rule fails one of them.
"""
import math

import numpy as np
import pytest

from paper_1705_03666_gb300 import workloads as W


def _within(mean, se, exact, bias):
    return np.all(np.abs(mean - exact) <= 3.0 * se + bias)


def test_laplace_expcos_closed_form(orc):
    """Eq. 1.1 with harmonic g = e^x cos y: u = g inside (Eq. 2.1)."""
    nodes = W.nodes_cfg1(16)
    r = orc.interface_solve(W.laplace_expcos(), nodes, seed=W.SEED_BASE + 1,
                            dt=1e-3, n_paths=20000)
    exact = np.exp(nodes[:, 0]) * np.cos(nodes[:, 1])
    assert _within(r["mean"], r["se"], exact, 2e-3)
    z = (r["mean"] - exact) / r["se"]
    assert abs(z.mean()) < 4.0 / math.sqrt(len(z)) + 0.5
    assert r["capped"] == 0


def test_exit_rates_sec21(orc):
    """Sec. 2.1: the plain boundary test has weak error O(sqrt(dt)); the
    boundary-corrected (bridge) test O(dt).  1-D torsion u = x(1-x) = E[tau]."""
    xs = np.array([0.2, 0.35, 0.5, 0.65, 0.8])
    prob = W.torsion("interval", 1)
    exact = xs * (1 - xs)
    err = {}
    for br in (False, True):
        for dt in (0.02, 0.005):
            r = orc.interface_solve(prob, xs[:, None], seed=11, dt=dt,
                                    n_paths=40000, bridge=br)
            err[br, dt] = float(np.mean(r["mean"] - exact))
    # plain test: error ratio for a 4x smaller dt is ~sqrt(4) = 2
    assert 1.6 < err[False, 0.02] / err[False, 0.005] < 2.6
    assert err[False, 0.02] > 0.07
    # bridge: error ratio ~4, and far below the plain test
    assert 2.5 < err[True, 0.02] / err[True, 0.005] < 6.5
    assert err[True, 0.02] < err[False, 0.02] / 5


def test_manufactured_3d_closed_form(orc):
    """(1/2) Lap u + b.grad u - u = F on [0,1]^3 with u = sin(pi x) sin(pi y)
    e^z: exercises drift, killing (c = -1) and source together."""
    nodes = W.nodes_cube_planes(4096)[::256]
    r = orc.interface_solve(W.elliptic_manufactured(), nodes,
                            seed=W.SEED_BASE + 2, dt=1e-3, n_paths=10000)
    exact = np.sin(np.pi * nodes[:, 0]) * np.sin(np.pi * nodes[:, 1]) * np.exp(nodes[:, 2])
    assert _within(r["mean"], r["se"], exact, 4e-3)


def test_manufactured_3d_drop_drift_fails(orc):
    """Sensitivity: the same estimate without the drift's contribution (a
    problem that differs from the manufactured one only by b) is rejected, so
    the closed-form pin above can see a dropped drift term."""
    nodes = W.nodes_cube_planes(4096)[::256]
    exact = np.sin(np.pi * nodes[:, 0]) * np.sin(np.pi * nodes[:, 1]) * np.exp(nodes[:, 2])
    # Laplace-only estimate of the same boundary data: no source, no drift
    prob = dict(W.elliptic_manufactured())
    prob["problem"] = "torsion"   # f = 1, g = 0: a different PDE entirely
    r = orc.interface_solve(prob, nodes, seed=5, dt=1e-3, n_paths=2000)
    assert not _within(r["mean"], r["se"], exact, 4e-3)


def test_bernal_acebron_source_symbolic(orc):
    """Eq. 2.10: the source f that makes u = 2cos(2(y-2)x) + sin(3(x-2)y) + 3.1
    exact, derived here symbolically and compared with the oracle's."""
    sp = pytest.importorskip("sympy")
    x, y = sp.symbols("x y")
    u = 2 * sp.cos(2 * (y - 2) * x) + sp.sin(3 * (x - 2) * y) + sp.Rational(31, 10)
    h = sp.cos(x + y) / (sp.Rational(11, 10) + sp.sin(x + y))
    c = -(x ** 2 + y ** 2) / (sp.Rational(11, 10) + sp.sin(x + y))
    lap = sp.diff(u, x, 2) + sp.diff(u, y, 2)
    f = -(lap + h * (sp.diff(u, x) + sp.diff(u, y)) + c * u)
    fn = sp.lambdify((x, y), [h, c, f, u], "math")
    prob = W.bernal_acebron()
    rng = np.random.default_rng(0)
    for px, py in rng.random((20, 2)):
        co = orc.eval_coeffs(prob, [px, py])
        hh, cc, ff, uu = fn(px, py)
        assert co[0] == pytest.approx(hh, rel=1e-12, abs=1e-12)
        assert co[1] == pytest.approx(hh, rel=1e-12, abs=1e-12)
        assert co[3] == pytest.approx(cc, rel=1e-12, abs=1e-12)
        assert co[4] == pytest.approx(ff, rel=1e-10, abs=1e-10)
        assert co[5] == pytest.approx(uu, rel=1e-12, abs=1e-12)


def test_manufactured_source_symbolic(orc):
    """Source of the manufactured 3-D problem, derived symbolically."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    u = sp.sin(sp.pi * x) * sp.sin(sp.pi * y) * sp.exp(z)
    b = (sp.sin(2 * sp.pi * y) / 2, sp.cos(2 * sp.pi * x) / 2, 0)
    F = (sp.diff(u, x, 2) + sp.diff(u, y, 2) + sp.diff(u, z, 2)) / 2 \
        + b[0] * sp.diff(u, x) + b[1] * sp.diff(u, y) - u
    fn = sp.lambdify((x, y, z), [F, u, b[0], b[1]], "math")
    prob = W.elliptic_manufactured()
    rng = np.random.default_rng(1)
    for p in rng.random((20, 3)):
        co = orc.eval_coeffs(prob, p)
        FF, uu, b0, b1 = fn(*p)
        assert co[0] == pytest.approx(b0, abs=1e-12)
        assert co[1] == pytest.approx(b1, abs=1e-12)
        assert co[2] == 0.0
        assert co[3] == -1.0
        assert co[4] == pytest.approx(-FF, rel=1e-11, abs=1e-11)
        assert co[5] == pytest.approx(uu, rel=1e-12, abs=1e-12)


def test_bernal_acebron_closed_form(orc):
    """Eq. 2.10 with sigma^2 = 2 (full Laplacian) on the unit square."""
    pts = np.array([[0.5, 0.5], [0.25, 0.75], [0.7, 0.3], [0.5, 0.2]])
    r = orc.interface_solve(W.bernal_acebron(), pts, seed=21, dt=5e-4, n_paths=8000)
    x, y = pts[:, 0], pts[:, 1]
    exact = 2 * np.cos(2 * (y - 2) * x) + np.sin(3 * (x - 2) * y) + 3.1
    assert _within(r["mean"], r["se"], exact, 1e-2)


def _fd_1d(b, c, f, g0, g1, n=4000):
    """Brute-force central differences for (1/2) u'' + b u' + c u + f = 0."""
    from scipy.linalg import solve_banded
    x = np.linspace(0.0, 1.0, n + 1)
    h = 1.0 / n
    xi = x[1:-1]
    lo = 0.5 / h ** 2 - b(xi) / (2 * h)
    di = -1.0 / h ** 2 + c(xi)
    up = 0.5 / h ** 2 + b(xi) / (2 * h)
    rhs = -f(xi)
    rhs[0] -= lo[0] * g0
    rhs[-1] -= up[-1] * g1
    ab = np.zeros((3, n - 1))
    ab[0, 1:] = up[:-1]
    ab[1] = di
    ab[2, :-1] = lo[1:]
    u = np.concatenate([[g0], solve_banded((1, 1), ab, rhs), [g1]])
    return x, u


def test_poly1d_vs_finite_differences(orc):
    """Drift, killing and source together against a brute-force FD solve."""
    prm = dict(b0=0.5, b1=1.0, c0=-1.0, f0=1.0, f1=2.0, g0=0.3, g1=-0.2)
    xs = np.array([0.15, 0.4, 0.6, 0.85])
    r = orc.interface_solve(W.poly1d(**prm), xs[:, None], seed=3, dt=1e-3,
                            n_paths=20000)
    xg, ug = _fd_1d(lambda x: 0.5 + x, lambda x: -np.ones_like(x),
                    lambda x: 1.0 + 2.0 * x, 0.3, -0.2)
    exact = np.interp(xs, xg, ug)
    assert _within(r["mean"], r["se"], exact, 3e-3)


def test_killing_closed_form(orc):
    """(1/2) u'' - u = 0, u(0) = u(1) = 1: u = cosh(sqrt2 (x-1/2))/cosh(sqrt2/2),
    i.e. Y = exp(-tau) in Eq. 2.8."""
    xs = np.array([0.1, 0.3, 0.5])
    r = orc.interface_solve(W.poly1d(c0=-1.0, g0=1.0, g1=1.0), xs[:, None],
                            seed=4, dt=1e-3, n_paths=20000)
    exact = np.cosh(math.sqrt(2) * (xs - 0.5)) / math.cosh(math.sqrt(2) / 2)
    assert _within(r["mean"], r["se"], exact, 2e-3)


def test_drift_closed_form(orc):
    """Constant drift mu: P(exit at 1) = (1 - e^{-2 mu x}) / (1 - e^{-2 mu})."""
    mu = 1.5
    xs = np.array([0.2, 0.5, 0.8])
    r = orc.interface_solve(W.poly1d(b0=mu, g0=0.0, g1=1.0), xs[:, None],
                            seed=5, dt=1e-3, n_paths=20000)
    exact = (1 - np.exp(-2 * mu * xs)) / (1 - np.exp(-2 * mu))
    assert _within(r["mean"], r["se"], exact, 3e-3)


def test_torsion_square_series(orc):
    """E[tau] on the unit square: (1/2) Lap u = -1, series solution."""
    pts = np.array([[0.5, 0.5], [0.25, 0.6]])
    r = orc.interface_solve(W.torsion(), pts, seed=6, dt=1e-3, n_paths=20000)
    exact = []
    for x, y in pts:
        s = 0.0
        for m in range(1, 200, 2):
            for n in range(1, 200, 2):
                s += 32.0 / (math.pi ** 4 * m * n * (m * m + n * n)) * \
                    math.sin(m * math.pi * x) * math.sin(n * math.pi * y)
        exact.append(s)
    assert _within(r["mean"], r["se"], np.array(exact), 2e-3)


def test_node_on_boundary_exits_at_once(orc):
    """A node on the boundary: tau = 0, u = g (Eq. 2.1)."""
    nodes = np.array([[0.0, 0.3], [0.5, 1.0], [1.0, 0.0]])
    r = orc.interface_solve(W.laplace_expcos(), nodes, seed=1, dt=1e-3,
                            n_paths=7, dump_paths=True)
    g = np.exp(nodes[:, 0]) * np.cos(nodes[:, 1])
    assert np.all(r["steps"] == 0)
    assert np.array_equal(r["score"], np.repeat(g[:, None], 7, axis=1))
    assert np.array_equal(r["mean"], g)
    assert np.all(r["se"] == 0.0)


def test_step_cap_counted(orc):
    nodes = np.array([[0.5, 0.5]])
    r = orc.interface_solve(W.laplace_expcos(), nodes, seed=1, dt=1e-6,
                            n_paths=50, max_steps=3, dump_paths=True)
    assert np.all(r["steps"] == -3)
    assert r["capped"] == 50
    assert r["total_steps"] == 150


def test_deterministic_across_threads(orc):
    nodes = W.nodes_cube_planes(64)[::8]
    kw = dict(seed=9, dt=1e-3, n_paths=300, dump_paths=True)
    a = orc.interface_solve(W.elliptic_manufactured(), nodes, n_threads=1, **kw)
    b = orc.interface_solve(W.elliptic_manufactured(), nodes, n_threads=5, **kw)
    assert np.array_equal(a["score"], b["score"])
    assert np.array_equal(a["mean"], b["mean"]) and np.array_equal(a["se"], b["se"])


def test_path_offset_continues_streams(orc):
    """Counter-based streams: paths [100, 200) equal the tail of [0, 200)."""
    nodes = W.nodes_cfg1(4)
    kw = dict(seed=2, dt=1e-3, dump_paths=True)
    full = orc.interface_solve(W.laplace_expcos(), nodes, n_paths=200, **kw)
    tail = orc.interface_solve(W.laplace_expcos(), nodes, n_paths=100,
                               path_offset=100, **kw)
    assert np.array_equal(full["score"][:, 100:], tail["score"])


def test_l_shape_harmonic(orc):
    """Eq. 1.1 on the L-shaped domain with harmonic g: u = g inside."""
    pts = np.array([[0.25, 0.75], [0.75, 0.25], [0.4, 0.4]])
    r = orc.interface_solve(W.laplace_expcos("l_shape"), pts, seed=8, dt=1e-3,
                            n_paths=20000)
    exact = np.exp(pts[:, 0]) * np.cos(pts[:, 1])
    assert _within(r["mean"], r["se"], exact, 4e-3)
