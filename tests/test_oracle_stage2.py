"""Pins for the oracle's deterministic stage (CPU only): the interface
interpolator and the subdomain solver of Sec. 2.1."""
import numpy as np

from paper_1705_03666_gb300 import workloads as W


def test_spline_reproduces_cubics(orc):
    """A not-a-knot cubic spline reproduces any cubic exactly."""
    p = np.polynomial.Polynomial([0.3, -1.2, 2.0, 0.7])
    s = W.nodes_cfg1(16)[:, 1]
    q = np.linspace(0, 1, 129)
    v = orc.spline_interface(s, p(s), q, p(0.0), p(1.0))
    np.testing.assert_allclose(v, p(q), rtol=0, atol=1e-12)


def test_spline_interpolates_and_converges(orc):
    s = W.nodes_cfg1(16)[:, 1]
    q = np.linspace(0, 1, 129)
    f = lambda y: np.exp(0.5) * np.cos(y)
    v = orc.spline_interface(s, f(s), s, f(0.0), f(1.0))
    np.testing.assert_allclose(v, f(s), atol=1e-14)
    err = np.max(np.abs(orc.spline_interface(s, f(s), q, f(0.0), f(1.0)) - f(q)))
    assert err < 1e-6


def test_stencil_tiny_dense(orc):
    """3x3 interior on a 5x5 grid against a hand-assembled dense system."""
    rng = np.random.default_rng(0)
    u = rng.standard_normal((5, 5))
    hx, hy = 0.25, 0.5
    out = orc.stencil_solve(u, (hx, hy))
    # residual of the 5-point operator on the interior is zero
    r = (out[1:-1, 2:] - 2 * out[1:-1, 1:-1] + out[1:-1, :-2]) / hx ** 2 \
        + (out[2:, 1:-1] - 2 * out[1:-1, 1:-1] + out[:-2, 1:-1]) / hy ** 2
    assert np.max(np.abs(r)) < 1e-10
    # boundary untouched
    assert np.array_equal(out[0], u[0]) and np.array_equal(out[:, -1], u[:, -1])
    # independent dense assembly
    idx = {(i, j): k for k, (i, j) in enumerate([(i, j) for i in range(1, 4) for j in range(1, 4)])}
    A = np.zeros((9, 9)); b = np.zeros(9)
    for (i, j), k in idx.items():
        A[k, k] = 2 / hx ** 2 + 2 / hy ** 2
        for (di, dj, w) in ((0, 1, hx), (0, -1, hx), (1, 0, hy), (-1, 0, hy)):
            q = (i + di, j + dj)
            if q in idx:
                A[k, idx[q]] -= 1 / w ** 2
            else:
                b[k] += u[q] / w ** 2
    sol = np.linalg.solve(A, b)
    np.testing.assert_allclose([out[i, j] for (i, j) in idx], sol, atol=1e-12)


def test_stencil_harmonic_second_order(orc):
    """Exact harmonic e^x cos y on [0, 1/2] x [0, 1]: error O(h^2)."""
    errs = []
    for n in (17, 33):
        x = np.linspace(0.0, 0.5, n)
        y = np.linspace(0.0, 1.0, n)
        X, Y = np.meshgrid(x, y)
        ex = np.exp(X) * np.cos(Y)
        u = ex.copy(); u[1:-1, 1:-1] = 0.0
        out = orc.stencil_solve(u, (0.5 / (n - 1), 1.0 / (n - 1)))
        errs.append(np.max(np.abs(out - ex)))
    assert 3.2 < errs[0] / errs[1] < 4.8
    assert errs[1] < 1e-4


def test_stencil_maximum_principle(orc):
    rng = np.random.default_rng(1)
    u = rng.random((9, 12))
    u[1:-1, 1:-1] = 10.0
    out = orc.stencil_solve(u, (0.1, 0.2))
    bnd = np.concatenate([u[0], u[-1], u[:, 0], u[:, -1]])
    assert out[1:-1, 1:-1].max() <= bnd.max() and out[1:-1, 1:-1].min() >= bnd.min()


# ---------------------------------------------------------------------------
# 3-D stage two: interface interpolation on the internal planes of the cube
# and the 7-point elliptic subdomain solve
# ---------------------------------------------------------------------------
def _exact3(x):
    return np.sin(np.pi * x[..., 0]) * np.sin(np.pi * x[..., 1]) * np.exp(x[..., 2])


def test_rbf_reproduces_linear_data_and_interpolates(orc):
    rng = np.random.default_rng(1)
    pts = rng.uniform(0, 1, (80, 2))
    q = rng.uniform(0, 1, (200, 2))
    lin = lambda p: 0.7 - 1.3 * p[:, 0] + 2.1 * p[:, 1]
    np.testing.assert_allclose(orc.rbf_interp(pts, lin(pts), q), lin(q), atol=1e-10)
    v = np.cos(3 * pts[:, 0]) * pts[:, 1]
    np.testing.assert_allclose(orc.rbf_interp(pts, v, pts), v, atol=1e-10)


def test_plane_interface_converges_on_smooth_data(orc):
    """The config's nodes on the plane x = 1/2 with exact values: the
    interpolant approaches the solution on the plane as nodes are added."""
    prob = W.elliptic_manufactured()
    nodes = W.nodes_cube_planes(4096)
    on = (np.arange(4096) % 3 == 0) & (nodes[:, 0] == 0.5)
    g = np.linspace(0.02, 0.98, 25)
    q = np.stack(np.meshgrid([0.5], g, g, indexing="ij"), -1).reshape(-1, 3)
    errs = []
    for k in (120, 455):
        sel = nodes[on][:k]
        v = orc.plane_interface(prob, 0, 0.5, sel, _exact3(sel), q)
        errs.append(np.max(np.abs(v - _exact3(q))))
    assert errs[1] < 2e-3 and errs[1] < 0.5 * errs[0], errs
    # boundary points carry g exactly
    b = orc.plane_boundary_points(0, 0.5, 8)
    v = orc.plane_interface(prob, 0, 0.5, nodes[on][:50], _exact3(nodes[on][:50]), b)
    np.testing.assert_allclose(v, _exact3(b), atol=1e-12)


def test_elliptic_box_solve_tiny_dense(orc):
    """2 x 2 x 2 interior unknowns: the sparse assembly against a dense one
    built point by point."""
    prob = W.elliptic_manufactured()
    lo, hi = (0.25, 0.5, 0.0), (0.5, 0.75, 0.25)
    rng = np.random.default_rng(2)
    ub = rng.standard_normal((4, 4, 4))
    out = orc.elliptic_box_solve(prob, ub, lo, hi)
    h = [(hi[a] - lo[a]) / 3 for a in range(3)]
    unk = [(k, j, i) for k in (1, 2) for j in (1, 2) for i in (1, 2)]
    A = np.zeros((8, 8))
    b = np.zeros(8)
    for r, (k, j, i) in enumerate(unk):
        x = np.array([lo[0] + i * h[0], lo[1] + j * h[1], lo[2] + k * h[2]])
        c = orc.eval_coeffs(prob, x)
        A[r, r] += c[3] - sum(1.0 / hh ** 2 for hh in h)
        b[r] -= c[4]
        for a, (di, dj, dk) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
            for sgn in (-1, 1):
                nb = (k + sgn * dk, j + sgn * dj, i + sgn * di)
                w = 0.5 / h[a] ** 2 + sgn * c[a] / (2 * h[a])
                if nb in unk:
                    A[r, unk.index(nb)] += w
                else:
                    b[r] -= w * ub[nb]
    sol = np.linalg.solve(A, b)
    np.testing.assert_allclose([out[p] for p in unk], sol, rtol=1e-12)
    mask = np.ones((4, 4, 4), bool)
    mask[1:3, 1:3, 1:3] = False
    assert np.array_equal(out[mask], ub[mask])


def test_elliptic_box_solve_second_order(orc):
    """The manufactured 3-D problem on a subdomain of the 4x4x4 split with
    exact Dirichlet data: the discrete solution converges at O(h^2) (a wrong
    drift sign, index or killing term would leave an O(1) error)."""
    prob = W.elliptic_manufactured()
    lo, hi = (0.25, 0.5, 0.75), (0.5, 0.75, 1.0)
    errs = []
    for n in (9, 17):
        t = [np.linspace(lo[a], hi[a], n) for a in range(3)]
        Z, Y, X = np.meshgrid(t[2], t[1], t[0], indexing="ij")
        ex = _exact3(np.stack([X, Y, Z], -1))
        ub = ex.copy()
        ub[1:-1, 1:-1, 1:-1] = 0.0
        errs.append(np.max(np.abs(orc.elliptic_box_solve(prob, ub, lo, hi) - ex)))
    assert errs[1] < 1e-4
    assert 3.5 < errs[0] / errs[1] < 4.5, errs
