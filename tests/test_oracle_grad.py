"""Pins for the oracle's derivative estimators (CPU only).

theta (linear boundary-data weights): the paths do not depend on theta, so the
pathwise derivative E[dg/dtheta(X_tau) Y_tau] is exact for the estimator and
equals a common-random-number central difference to rounding.
phi (drift weights): likelihood-ratio estimator of the discrete scheme, pinned
against derivatives of a brute-force finite-difference PDE solve in 1-D
(strong pin) and against common-random-number finite differences of the 2-D
Poisson-Fourier workload (statistical pin).
"""
import numpy as np
import pytest

from paper_1705_03666_gb300 import workloads as W
from test_oracle_paths import _fd_1d


def _fdsolve(p, xs):
    xg, ug = _fd_1d(lambda x: p["b0"] + p["b1"] * x, lambda x: p["c0"] + 0 * x,
                    lambda x: p["f0"] + p["f1"] * x, p["g0"], p["g1"])
    return np.interp(xs, xg, ug)


def test_1d_derivatives_vs_fd_solve(orc):
    prm = dict(b0=0.8, b1=0.5, c0=-0.5, f0=1.0, f1=0.0, g0=0.2, g1=1.0)
    xs = np.array([0.3, 0.6])
    J, Jse = orc.interface_jacobian(W.poly1d(**prm), xs[:, None], seed=12,
                                    dt=1e-3, n_paths=40000)
    ref = []
    for k in ("g0", "g1", "b0", "b1"):
        pp, pm = dict(prm), dict(prm)
        pp[k] += 1e-3
        pm[k] -= 1e-3
        ref.append((_fdsolve(pp, xs) - _fdsolve(pm, xs)) / 2e-3)
    ref = np.array(ref).T
    assert np.all(np.abs(J - ref) <= 3.0 * Jse + 2e-3)


def test_theta_derivative_is_crn_difference(orc):
    prob = W.poisson_fourier(5)
    nodes = W.nodes_cfg5(512)[::256]
    kw = dict(seed=W.SEED_BASE + 5, dt=1e-3, n_paths=2000)
    J, _ = orc.interface_jacobian(prob, nodes, **kw)
    h = 1e-3
    for k in (0, 9, 27, 63):
        pp, pm = dict(prob), dict(prob)
        pp["params"] = prob["params"].copy(); pp["params"][k] += h
        pm["params"] = prob["params"].copy(); pm["params"][k] -= h
        d = (orc.interface_solve(pp, nodes, **kw)["mean"]
             - orc.interface_solve(pm, nodes, **kw)["mean"]) / (2 * h)
        np.testing.assert_allclose(d, J[:, k], rtol=1e-7, atol=1e-9)


def test_theta_linearity_reconstructs_estimate(orc):
    """u = sum_k theta_k J_k + E[tau]: with theta = 0 the estimate is E[tau]."""
    prob = W.poisson_fourier(5)
    nodes = W.nodes_cfg5(512)[::256]
    kw = dict(seed=3, dt=1e-3, n_paths=1000)
    J, _ = orc.interface_jacobian(prob, nodes, **kw)
    u = orc.interface_solve(prob, nodes, **kw)["mean"]
    p0 = dict(prob)
    p0["params"] = prob["params"].copy(); p0["params"][:64] = 0.0
    tau = orc.interface_solve(p0, nodes, **kw)["mean"]
    np.testing.assert_allclose(J[:, :64] @ prob["params"][:64] + tau, u,
                               rtol=1e-10, atol=1e-10)


def test_phi_lr_vs_crn_finite_difference(orc):
    prob = W.poisson_fourier(5)
    nodes = W.nodes_cfg5(512)[::128]
    kw = dict(seed=W.SEED_BASE + 5, dt=1e-3, n_paths=20000)
    J, Jse = orc.interface_jacobian(prob, nodes, **kw)
    h = 0.05
    zs = []
    for j in (0, 9):
        pp, pm = dict(prob), dict(prob)
        pp["params"] = prob["params"].copy(); pp["params"][64 + j] += h
        pm["params"] = prob["params"].copy(); pm["params"][64 + j] -= h
        sp = orc.interface_solve(pp, nodes, dump_paths=True, **kw)["score"]
        sm = orc.interface_solve(pm, nodes, dump_paths=True, **kw)["score"]
        d = (sp - sm) / (2 * h)
        fd, fse = d.mean(1), d.std(1) / np.sqrt(d.shape[1])
        zs.append((fd - J[:, 64 + j]) / np.sqrt(fse ** 2 + Jse[:, 64 + j] ** 2))
    z = np.concatenate(zs)
    assert np.max(np.abs(z)) < 4.0
    assert np.mean(z ** 2) < 2.5
