"""Seeded synthetic workloads for the PDD interface-node Monte Carlo.

This module holds input generators only: node placements, coefficient
parameters and seeds.  It contains none of the method's arithmetic, imports
nothing else from the package, and is the one module that both the CUDA path
(through the Python binding) and the CPU oracle consume.

Problems are plain dicts with string names, so neither side shares a constant
with the other:

  problem   laplace_expcos | elliptic_manufactured | poisson_fourier |
            bernal_acebron | poly1d | torsion | kpp
  geometry  interval | unit_square | l_shape | unit_cube | free_space
  dim, sigma, params (float64 array)

The five workloads follow the paper's settings where it gives them (the 2-D
Laplace problem of Eq. 1.1 with harmonic data, the KPP example of Sec. 3.1.1
with N = 1e5 samples per node and time points T_i on an interface grid) and
fixed synthetic choices elsewhere; every choice is listed next to it.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 0x1705036660000000

# Plastic number: real root of x^3 = x + 1 (generator of the R2 sequence).
_PLASTIC = 1.3247179572447460259609088544780973407344


def r2_points(count: int, offset: float = 0.5) -> np.ndarray:
    """The R2 low-discrepancy sequence in [0,1)^2: frac(offset + k*(1/p, 1/p^2))."""
    k = np.arange(count, dtype=np.float64)[:, None]
    a = np.array([1.0 / _PLASTIC, 1.0 / _PLASTIC ** 2])
    return np.mod(offset + k * a, 1.0)


# --------------------------------------------------------------------------
# Problems
# --------------------------------------------------------------------------
def _robin(reflect, phi: float) -> np.ndarray:
    """Optional reflecting faces: [mask, phi] with bit j of the mask for face
    j = 2k + s of the box (x_k = s), Robin condition du/dN = phi u + psi."""
    if not reflect:
        return np.zeros(0)
    mask = 0
    for j in reflect:
        mask |= 1 << int(j)
    return np.array([float(mask), float(phi)])


def laplace_expcos(geometry: str = "unit_square", reflect=None, phi: float = 0.0) -> dict:
    """Eq. 1.1 on the unit square (or L-shape) with harmonic g = e^x cos y;
    faces listed in `reflect` carry Robin data du/dN = phi u + psi with psi
    chosen so that e^x cos y stays exact (Eq. 2.4)."""
    return {"problem": "laplace_expcos", "geometry": geometry, "dim": 2,
            "sigma": 1.0, "params": _robin(reflect, phi)}


def elliptic_manufactured(reflect=None, phi: float = 0.0) -> dict:
    """(1/2) Lap u + b.grad u - u = F on [0,1]^3, b = (0.5 sin 2 pi y,
    0.5 cos 2 pi x, 0), F manufactured from u = sin(pi x) sin(pi y) e^z;
    optional reflecting faces with Robin data that keep u exact."""
    return {"problem": "elliptic_manufactured", "geometry": "unit_cube",
            "dim": 3, "sigma": 1.0, "params": _robin(reflect, phi)}


def poisson_fourier(seed: int = 5, phi_scale: float = 0.1) -> dict:
    """(1/2) Lap u + b_phi.grad u = -1 on [0,1]^2 with boundary data
    g_theta = sum_{m,n<8} theta_mn cos(m pi x) cos(n pi y) and drift
    b_phi = (sum_j phi_j sin(j pi y), sum_j phi_{8+j} sin(j pi x)), j = 1..8.
    theta ~ N(0,1), phi ~ phi_scale * N(0,1), drawn with numpy seed `seed`."""
    rng = np.random.default_rng(seed)
    theta = rng.standard_normal(64)
    phi = phi_scale * rng.standard_normal(16)
    return {"problem": "poisson_fourier", "geometry": "unit_square", "dim": 2,
            "sigma": 1.0, "params": np.concatenate([theta, phi])}


def bernal_acebron() -> dict:
    """Eq. 2.10 (full Laplacian, so sigma^2 = 2) on the unit square standing in
    for the lost Fig. 2.1 domain; exact u printed with Eq. 2.10."""
    return {"problem": "bernal_acebron", "geometry": "unit_square", "dim": 2,
            "sigma": float(np.sqrt(2.0)), "params": np.zeros(0)}


def poly1d(b0=0.0, b1=0.0, c0=0.0, f0=0.0, f1=0.0, g0=0.0, g1=0.0) -> dict:
    """1-D test family on (0,1): (1/2) u'' + (b0 + b1 x) u' + c0 u + f0 + f1 x = 0,
    u(0) = g0, u(1) = g1."""
    return {"problem": "poly1d", "geometry": "interval", "dim": 1, "sigma": 1.0,
            "params": np.array([b0, b1, c0, f0, f1, g0, g1], dtype=np.float64)}


def torsion(geometry: str = "unit_square", dim: int = 2, reflect=None, phi: float = 0.0) -> dict:
    """(1/2) Lap u = -1, u = 0 on the boundary: u(x) = E[tau]; faces in
    `reflect` carry du/dN = phi u instead."""
    return {"problem": "torsion", "geometry": geometry, "dim": dim, "sigma": 1.0,
            "params": _robin(reflect, phi)}


def kpp(psi: str = "sigmoid", psi_param: float = 4.0, beta: float = 1.0,
        q=(0.0, 0.0, 1.0), alpha=None, dim: int = 2, geometry: str = "free_space") -> dict:
    """u_t = (1/2) Lap u + beta (sum_k alpha_k u^k - u), u(.,0) = psi (Eq. 3.1,
    Sec. 3.2 when alpha != q).  psi in {const, sigmoid, travelling, sine}:
    const c; 1/(1+exp(-a x1)); 1 - (1+exp(a x1))^-2; prod_k sin(pi x_k).
    A bounded geometry (interval, unit_square, l_shape) adds absorbing
    boundaries with data g(x, s) fixed by the psi kind (Eq. 3.2)."""
    q = np.asarray(q, dtype=np.float64)
    alpha = q.copy() if alpha is None else np.asarray(alpha, dtype=np.float64)
    K = len(q) - 1
    kind = {"const": 0.0, "sigmoid": 1.0, "travelling": 2.0, "sine": 3.0}[psi]
    params = np.concatenate([[beta, kind, psi_param, float(K)], q, alpha])
    return {"problem": "kpp", "geometry": geometry, "dim": dim, "sigma": 1.0,
            "params": params}


# --------------------------------------------------------------------------
# Node placements
# --------------------------------------------------------------------------
def nodes_cfg1(count: int = 16) -> np.ndarray:
    """Equispaced interface nodes on x = 1/2, y_k = k/(count+1), k = 1..count
    (the end points lie on the boundary, where u = g is known)."""
    y = np.arange(1, count + 1, dtype=np.float64) / (count + 1)
    return np.stack([np.full_like(y, 0.5), y], axis=1)


def nodes_cube_planes(count: int = 4096) -> np.ndarray:
    """Nodes on the 9 internal planes of a 4x4x4 split of [0,1]^3: node n lies
    on axis a = n mod 3, plane x_a = (j+1)/4 with j = (n div 3) mod 3; its other
    two coordinates are R2 point n div 9."""
    n = np.arange(count)
    a = n % 3
    j = (n // 3) % 3
    pts = r2_points(int(n.max()) // 9 + 1 if count else 0)[n // 9]
    out = np.zeros((count, 3))
    for axis in range(3):
        sel = a == axis
        others = [k for k in range(3) if k != axis]
        out[sel, axis] = (j[sel] + 1) / 4.0
        out[sel, others[0]] = pts[sel, 0]
        out[sel, others[1]] = pts[sel, 1]
    return out


def nodes_kpp(lines=(-3.0, -1.0, 1.0, 3.0), n_x2: int = 16, n_t: int = 16,
              t_max: float = 1.0) -> np.ndarray:
    """Space-time interface nodes (x1, x2, t): interface lines x1 in `lines`,
    x2 in linspace(-2, 2, n_x2), t = T_i = i t_max / n_t, i = 1..n_t
    (Algorithm 3.1 evaluates each interface node at a series of times)."""
    out = []
    for x1 in lines:
        for x2 in np.linspace(-2.0, 2.0, n_x2):
            for i in range(1, n_t + 1):
                out.append((x1, x2, i * t_max / n_t))
    return np.array(out, dtype=np.float64)


def nodes_cfg5(per_line: int = 512, lines=(0.2, 0.4, 0.6, 0.8)) -> np.ndarray:
    """Interface lines x in `lines`, y_k = k/(per_line+1)."""
    y = np.arange(1, per_line + 1, dtype=np.float64) / (per_line + 1)
    return np.concatenate([np.stack([np.full_like(y, x), y], axis=1) for x in lines])


# --------------------------------------------------------------------------
# The five workloads
# --------------------------------------------------------------------------
def workload(k: int) -> dict:
    """Workload k in 1..5 (sizes at full scale)."""
    if k == 1:
        return {"name": "laplace2d_square_16nodes_1e4paths_dt1e-3_fp64",
                "prob": laplace_expcos(), "nodes": nodes_cfg1(16),
                "seed": SEED_BASE + 1, "dt": 1e-3, "n_paths": 10_000,
                "precision": "fp64", "bridge": True}
    if k == 2:
        return {"name": "elliptic3d_cube_4096nodes_1e5paths_dt1e-4_fp32",
                "prob": elliptic_manufactured(), "nodes": nodes_cube_planes(4096),
                "seed": SEED_BASE + 2, "dt": 1e-4, "n_paths": 100_000,
                "precision": "fp32", "bridge": True}
    if k == 3:
        mix = batch_mix()
        return {"name": "batch_square7000_lshape7000_cube6000_adaptive_se1e-4",
                **mix, "seed": SEED_BASE + 3, "n_pilot": 1000, "n_min": 1000,
                "n_max": 1_000_000, "target_se": 1e-4}
    if k == 4:
        return {"name": "kpp2d_1024nodes_1e5trees_beta1",
                "prob": kpp("sigmoid", 4.0, 1.0), "nodes": nodes_kpp(),
                "seed": SEED_BASE + 4, "n_trees": 100_000,
                "max_particles": 4096, "max_depth": 64}
    if k == 5:
        return {"name": "poisson2d_fourier_2048nodes_1e5paths_dt1e-3",
                "prob": poisson_fourier(5), "nodes": nodes_cfg5(512),
                "seed": SEED_BASE + 5, "dt": 1e-3, "n_paths": 100_000,
                "precision": "fp32", "bridge": True}
    raise ValueError(f"no workload {k}")


def kpp_bounded_square(n_trees: int = 100_000) -> dict:
    """Eq. 3.2 on the unit square: u_t = (1/2) Lap u + beta (u^2 - u) with
    beta = 4, psi and boundary data from the travelling wave
    1 - (1 + e^{a x - 5 beta t / 6})^-2, a = sqrt(beta / 3) (exact solution);
    nodes on the interfaces x in {1/4, 1/2, 3/4}, y = k/17 (k = 1..16), 16
    grid times T_i = i/16 scored by one tree per sample, dt = 1e-3."""
    beta = 4.0
    y = np.arange(1, 17, dtype=np.float64) / 17.0
    nodes = np.concatenate([np.stack([np.full_like(y, x), y], 1) for x in (0.25, 0.5, 0.75)])
    return {"name": "kpp_bounded_square_48nodes_16times_1e5trees_beta4_dt1e-3",
            "prob": kpp("travelling", float(np.sqrt(beta / 3.0)), beta, geometry="unit_square"),
            "nodes": nodes, "times": np.arange(1, 17, dtype=np.float64) / 16.0,
            "seed": SEED_BASE + 6, "n_trees": n_trees, "dt": 1e-3}


def nodes_lshape_interfaces(count: int) -> np.ndarray:
    """Nodes on the L-shape's interfaces: alternately on x = 1/2, y in (0, 1/2)
    and on y = 1/2, x in (0, 1/2), equispaced along each segment (the two
    artificial interfaces that cut the L into three squares)."""
    a = (count + 1) // 2
    b = count - a
    ya = np.arange(1, a + 1, dtype=np.float64) / (2 * (a + 1))
    xb = np.arange(1, b + 1, dtype=np.float64) / (2 * (b + 1))
    pts = np.concatenate([np.stack([np.full_like(ya, 0.5), ya], 1),
                          np.stack([xb, np.full_like(xb, 0.5)], 1)])
    return pts


def batch_mix(square: int = 7000, lshape: int = 7000, cube: int = 6000, seed: int = 3) -> dict:
    """The heterogeneous batch: Laplace on the unit square (interface x = 1/2),
    Laplace on the L-shape (its two interfaces), and the 3-D elliptic problem
    (internal planes of the cube); per-node dt drawn from {1e-3, 1e-4} with
    NumPy seed `seed`.  Returns problems, nodes [n, 3], problem index, dt."""
    rng = np.random.default_rng(seed)
    sq = np.stack([np.full(square, 0.5), np.arange(1, square + 1) / (square + 1)], 1)
    ls = nodes_lshape_interfaces(lshape)
    cb = nodes_cube_planes(cube)
    nodes = np.zeros((square + lshape + cube, 3))
    nodes[:square, :2] = sq
    nodes[square:square + lshape, :2] = ls
    nodes[square + lshape:] = cb
    pidx = np.concatenate([np.zeros(square), np.ones(lshape), np.full(cube, 2)]).astype(np.int32)
    dt = np.where(rng.random(len(nodes)) < 0.5, 1e-3, 1e-4)
    return {"problems": [laplace_expcos("unit_square"), laplace_expcos("l_shape"),
                         elliptic_manufactured()],
            "nodes": nodes, "problem_index": pidx, "dt": dt}


def every_kth_node(nodes: np.ndarray, k: int) -> np.ndarray:
    """Fixed subset of nodes (indices 0, k, 2k, ...)."""
    return np.ascontiguousarray(nodes[::k])
