"""Pins for the oracle's reflecting (Neumann/Robin) faces: the mixed BVP of
Eq. 2.4 with the local-time terms of Eq. 2.9 (-N dxi in X, phi Y dxi in Y,
psi Y dxi in Z), simulated with Lepingle's half-space reflection.  Closed
forms: 1-D torsion with a Neumann or Robin end, the harmonic e^x cos y with
Neumann and Robin faces, the 3-D manufactured solution with Robin faces."""
import numpy as np

from paper_1705_03666_gb300 import workloads as W


def test_torsion_1d_neumann_and_robin(orc):
    """(1/2) u'' = -1 on (0,1), u(0) = 0, u'(1) = phi u(1): u = -x^2 + A x
    with A = (2 - phi) / (1 - phi) (phi = 0: 2x - x^2)."""
    x = np.array([[0.2], [0.5], [0.8], [1.0]])
    for phi in (0.0, -1.0):
        r = orc.interface_solve(W.torsion("interval", 1, reflect=[1], phi=phi), x, seed=1,
                                dt=1e-3, n_paths=20000, bridge=True)
        A = (2 - phi) / (1 - phi)
        exact = -x[:, 0] ** 2 + A * x[:, 0]
        assert np.all(np.abs(r["mean"] - exact) < 4.5 * r["se"] + 3e-3), (phi, r["mean"], exact)


def test_torsion_1d_robin_differs_from_neumann(orc):
    x = np.array([[0.8]])
    a = orc.interface_solve(W.torsion("interval", 1, reflect=[1], phi=0.0), x, seed=2, dt=1e-3,
                            n_paths=20000)
    b = orc.interface_solve(W.torsion("interval", 1, reflect=[1], phi=-1.0), x, seed=2, dt=1e-3,
                            n_paths=20000)
    # exact: 0.96 and 0.56
    assert a["mean"][0] - b["mean"][0] > 0.3


def test_laplace_neumann_and_robin_faces(orc):
    """e^x cos y stays exact with face y = 0 Neumann (its normal derivative
    vanishes there) and face x = 1 Robin with phi = -2, psi = 3 e cos y."""
    nodes = np.array([[0.5, 0.5], [0.9, 0.2], [0.3, 0.05], [0.5, 0.0], [0.95, 0.9]])
    exact = np.exp(nodes[:, 0]) * np.cos(nodes[:, 1])
    for reflect, phi in (([2], 0.0), ([1], -2.0), ([1, 2], -2.0)):
        prob = W.laplace_expcos(reflect=reflect, phi=phi)
        r = orc.interface_solve(prob, nodes, seed=3, dt=1e-3, n_paths=20000, bridge=True)
        assert np.all(np.abs(r["mean"] - exact) < 4.5 * r["se"] + 4e-3), (reflect, r["mean"] - exact)


def test_start_on_reflecting_face_walks(orc):
    prob = W.laplace_expcos(reflect=[2])
    r = orc.interface_solve(prob, np.array([[0.5, 0.0]]), seed=4, dt=1e-3, n_paths=200,
                            dump_paths=True)
    assert np.all(r["steps"] > 0)
    r = orc.interface_solve(W.laplace_expcos(), np.array([[0.5, 0.0]]), seed=4, dt=1e-3,
                            n_paths=20, dump_paths=True)
    assert np.all(r["steps"] == 0)


def test_elliptic_3d_robin_faces(orc):
    """Manufactured u = sin(pi x) sin(pi y) e^z with face z = 0 Robin
    (phi = -1, where psi = 0) and face x = 0 Neumann (psi = -pi sin(pi y))."""
    nodes = np.array([[0.5, 0.5, 0.1], [0.1, 0.5, 0.5], [0.3, 0.7, 0.25]])
    prob = W.elliptic_manufactured(reflect=[4, 0], phi=-1.0)
    r = orc.interface_solve(prob, nodes, seed=5, dt=1e-3, n_paths=20000, bridge=True)
    exact = np.sin(np.pi * nodes[:, 0]) * np.sin(np.pi * nodes[:, 1]) * np.exp(nodes[:, 2])
    assert np.all(np.abs(r["mean"] - exact) < 4.5 * r["se"] + 5e-3), r["mean"] - exact
