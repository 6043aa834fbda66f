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
