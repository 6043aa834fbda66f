"""FP64 CPU oracle for the PDD interface-node Monte Carlo (arXiv:1705.03666).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference legs import this package.  The product
library never imports, links or calls it, and it imports nothing from the
product: it is a ctypes wrapper around ``oracle.c`` (plain C, double
precision) plus a few plain NumPy/SciPy routines for the deterministic stage of
the method (the interface interpolation and the subdomain solve, Sec. 2.1).

Each function cites the passage it follows.  Problems are described by the
plain dictionaries that ``paper_1705_03666_gb300.workloads`` builds (names, not
library enums), so that no constant is shared with the CUDA path.

Parity status per function (what pins it is listed in the tests):
  interface_solve    pinned (closed forms, FD brute force, invariants)
  interface_jacobian pinned (linearity in theta; CRN finite differences)
  branching_solve    pinned (ODE closed forms, travelling wave, CN solve)
  wos_solve          pinned (harmonic data, O(eps) bias, boundary nodes)
  branching_grid_solve pinned (KPP ODE with matching boundary data, travelling
                     wave, heat mode, bridge bias, marked law at every T_i)
  mlmc_level         pinned (harmonic telescoping sum, coarse = previous
                     level's law under a biased dt, level 0, variance decay)
  interface_solve with reflecting faces pinned (1-D Neumann/Robin torsion,
                     harmonic data with Neumann/Robin faces, 3-D Robin)
  spline_interface   pinned (reproduces cubics exactly; library routine)
  subdomain_solve    pinned (dense solve, exact harmonic at O(h^2))
  plane_interface    pinned (reproduces linear data exactly, interpolates at
                     the nodes, converges for smooth data; library routine)
  elliptic_box_solve pinned (dense assembly on a tiny grid, exact for a
                     quadratic with constant drift, O(h^2) to the manufactured
                     3-D solution)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

GEOMETRY = {"interval": 0, "unit_square": 1, "l_shape": 2, "unit_cube": 3,
            "free_space": 4}
PROBLEM = {"laplace_expcos": 1, "elliptic_manufactured": 2,
           "poisson_fourier": 3, "bernal_acebron": 4, "poly1d": 5,
           "torsion": 6, "kpp": 7}
PSI = {"const": 0, "sigmoid": 1, "travelling": 2}


class _Problem(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("geometry", ctypes.c_int32),
                ("dim", ctypes.c_int32), ("n_params", ctypes.c_int32),
                ("params", ctypes.POINTER(ctypes.c_double)),
                ("sigma", ctypes.c_double)]


class _MC(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("dt", ctypes.c_double),
                ("n_paths", ctypes.c_int64), ("max_steps", ctypes.c_int64),
                ("bridge", ctypes.c_int32), ("n_threads", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into liborc.so (no FMA contraction, so the
    host results are the same on x86-64 and aarch64)."""
    if force or not os.path.exists(_LIB) or \
            os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11",
                               "-D_GNU_SOURCE", "-shared", "-fPIC", "-o", tmp,
                               _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P, M = ctypes.POINTER(_Problem), ctypes.POINTER(_MC)
            dp = ctypes.POINTER(ctypes.c_double)
            lp = ctypes.POINTER(ctypes.c_int64)
            ip = ctypes.POINTER(ctypes.c_int32)
            up = ctypes.POINTER(ctypes.c_uint32)
            lib.orc_philox4x32_10.argtypes = [up, up, up]
            lib.orc_philox_stream.argtypes = [ctypes.c_uint64, ctypes.c_uint32,
                                              ctypes.c_uint32, ctypes.c_uint32,
                                              ctypes.c_uint32, ctypes.c_int64, up]
            lib.orc_eval_coeffs.argtypes = [P, dp, dp]
            lib.orc_eval_coeffs_many.argtypes = [P, dp, ctypes.c_int64, dp]
            lib.orc_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32,
                                        ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_int64, dp, dp]
            lib.orc_philox_constants.argtypes = [up]
            lib.orc_interface_solve.argtypes = [P, dp, ctypes.c_int64, lp, M,
                                                ctypes.c_int64, dp, dp, lp, dp,
                                                ip, dp, lp, lp]
            lib.orc_interface_solve.restype = ctypes.c_int
            lib.orc_interface_jacobian.argtypes = [P, dp, ctypes.c_int64, M, dp, dp, dp, ip]
            lib.orc_interface_jacobian.restype = ctypes.c_int
            lib.orc_jacobian_width.argtypes = [P]
            lib.orc_jacobian_width.restype = ctypes.c_int
            lib.orc_wos_solve.argtypes = [P, dp, ctypes.c_int64, lp, M, ctypes.c_double,
                                          dp, dp, lp, dp, ip, lp, dp]
            lib.orc_wos_solve.restype = ctypes.c_int
            lib.orc_branching_solve.argtypes = [P, dp, ctypes.c_int64, M,
                                                ctypes.c_int64, ctypes.c_int32,
                                                dp, dp, lp, lp, dp, ip]
            lib.orc_branching_solve.restype = ctypes.c_int
            lib.orc_branching_grid_solve.argtypes = [P, dp, ctypes.c_int64, dp, ctypes.c_int32,
                                                     M, ctypes.c_int64, ctypes.c_int32,
                                                     dp, dp, lp, lp, dp, ip]
            lib.orc_branching_grid_solve.restype = ctypes.c_int
            lib.orc_mlmc_level.argtypes = [P, dp, ctypes.c_int64, M, ctypes.c_int32,
                                           ctypes.c_int32, dp, dp, dp, dp, dp, ip, lp, dp]
            lib.orc_mlmc_level.restype = ctypes.c_int
            lib.orc_grid_ticks_per_unit.argtypes = [ctypes.c_double]
            lib.orc_grid_ticks_per_unit.restype = ctypes.c_double
            _lib = lib
    return _lib


def _ptr(a, ct):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _problem(prob: dict):
    params = np.ascontiguousarray(prob.get("params", np.zeros(0)), dtype=np.float64)
    if params.size == 0:
        params = np.zeros(1)
    s = _Problem(PROBLEM[prob["problem"]], GEOMETRY[prob["geometry"]],
                 int(prob["dim"]), int(params.size), _ptr(params, ctypes.c_double),
                 float(prob.get("sigma", 1.0)))
    return s, params  # keep params alive


def _mc(seed, dt, n_paths, max_steps, bridge, n_threads):
    return _MC(int(seed) & (2**64 - 1), float(dt), int(n_paths), int(max_steps),
               int(bool(bridge)), int(n_threads or os.cpu_count() or 1))


def philox4x32_10(ctr, key):
    """One Philox4x32-10 block (Salmon et al., SC'11)."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                          _ptr(out, ctypes.c_uint32))
    return out


def philox_stream(seed, j0, c1, c2, c3, n_blocks):
    """Blocks Philox((j0+b, c1, c2, c3), key=seed) for b < n_blocks, as u32[n,4]."""
    lib = _load()
    out = np.zeros((int(n_blocks), 4), dtype=np.uint32)
    lib.orc_philox_stream(int(seed), int(j0), int(c1), int(c2), int(c3),
                          int(n_blocks), _ptr(out, ctypes.c_uint32))
    return out


def normals(seed, n_pairs, c1=0, c2=0, c3=9):
    """2*n_pairs Box-Muller normals and n_pairs uniforms from Philox blocks
    (j, c1, c2, c3), j < n_pairs (same maps the estimators use)."""
    lib = _load()
    z = np.zeros(2 * int(n_pairs))
    u = np.zeros(int(n_pairs))
    lib.orc_normals(int(seed), int(c1), int(c2), int(c3), int(n_pairs),
                    _ptr(z, ctypes.c_double), _ptr(u, ctypes.c_double))
    return z, u


def philox_constants():
    """(M0, M1, W0, W1) used by the oracle's Philox."""
    lib = _load()
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox_constants(_ptr(out, ctypes.c_uint32))
    return [int(v) for v in out]


def eval_coeffs(prob: dict, x) -> np.ndarray:
    """(b0, b1, b2, c, f, g) of the problem at x, in the paper's form
    (1/2) sigma^2 Lap u + b.grad u + c u + f = 0 (Eq. 2.3-2.4)."""
    lib = _load()
    P, keep = _problem(prob)
    xx = np.zeros(3)
    xx[:len(x)] = x
    out = np.zeros(6)
    lib.orc_eval_coeffs(ctypes.byref(P), _ptr(xx, ctypes.c_double),
                        _ptr(out, ctypes.c_double))
    return out


def eval_coeffs_many(prob: dict, x) -> np.ndarray:
    """(b0, b1, b2, c, f, g) of the problem at points x [n, d] -> [n, 6]."""
    lib = _load()
    P, keep = _problem(prob)
    x = np.asarray(x, dtype=np.float64)
    xx = np.zeros((x.shape[0], 3))
    xx[:, :x.shape[1]] = x
    out = np.zeros((x.shape[0], 6))
    lib.orc_eval_coeffs_many(ctypes.byref(P), _ptr(xx, ctypes.c_double), x.shape[0],
                             _ptr(out, ctypes.c_double))
    return out


def interface_solve(prob: dict, nodes, *, seed, dt, n_paths, max_steps=10**7,
                    bridge=True, n_threads=None, path_offset=0,
                    dump_paths=False, node_ids=None):
    """Monte Carlo estimate of u at each node (Eq. 2.1-2.9, Sec. 2.1 numerics).

    node_ids (optional) gives the node index each node's random streams use
    (default: its position), so a subset of a large node list can be
    recomputed on the same streams.  Returns a dict with mean, se, n (per
    node), total_steps, capped, and, when dump_paths, score[n, N],
    steps[n, N] and exit[n, N, dim] (exit point) per path."""
    lib = _load()
    nodes = np.ascontiguousarray(nodes, dtype=np.float64).reshape(-1, int(prob["dim"]))
    n = nodes.shape[0]
    P, keep = _problem(prob)
    M = _mc(seed, dt, n_paths, max_steps, bridge, n_threads)
    mean, se = np.zeros(n), np.zeros(n)
    npaths = np.zeros(n, dtype=np.int64)
    score = np.zeros((n, n_paths)) if dump_paths else None
    steps = np.zeros((n, n_paths), dtype=np.int32) if dump_paths else None
    xexit = np.zeros((n, n_paths, int(prob["dim"]))) if dump_paths else None
    ts, tc = ctypes.c_int64(0), ctypes.c_int64(0)
    ids = None if node_ids is None else np.ascontiguousarray(node_ids, dtype=np.int64)
    if ids is not None and ids.shape != (n,):
        raise ValueError("node_ids must have one entry per node")
    rc = lib.orc_interface_solve(ctypes.byref(P), _ptr(nodes, ctypes.c_double), n,
                                 _ptr(ids, ctypes.c_int64),
                                 ctypes.byref(M), int(path_offset),
                                 _ptr(mean, ctypes.c_double), _ptr(se, ctypes.c_double),
                                 _ptr(npaths, ctypes.c_int64),
                                 _ptr(score, ctypes.c_double),
                                 _ptr(steps, ctypes.c_int32), _ptr(xexit, ctypes.c_double),
                                 ctypes.byref(ts), ctypes.byref(tc))
    if rc != 0:
        raise ValueError("oracle interface_solve: invalid arguments")
    out = {"mean": mean, "se": se, "n": npaths, "total_steps": ts.value,
           "capped": tc.value}
    if dump_paths:
        out["score"], out["steps"], out["exit"] = score, steps, xexit
    return out


def interface_jacobian(prob: dict, nodes, *, seed, dt, n_paths, max_steps=10**7,
                       bridge=True, n_threads=None, dump_paths=False):
    """Per-node derivatives of u w.r.t. the family's parameters: theta (linear
    boundary data, exact pathwise) then phi (drift, likelihood ratio).
    Poisson-Fourier: [n, 64 + 16]; poly1d: [n, 2 + 2] for (g0, g1, b0, b1).
    Returns (jac, jac_se), or with dump_paths (jac, jac_se, rec, steps): rec
    is [n, N, 4 + n_phi] per path (score, exit point x, y, z, L_1..L_nphi)."""
    lib = _load()
    d = int(prob["dim"])
    nodes = np.ascontiguousarray(nodes, dtype=np.float64).reshape(-1, d)
    n = nodes.shape[0]
    P, keep = _problem(prob)
    W = lib.orc_jacobian_width(ctypes.byref(P))
    M = _mc(seed, dt, n_paths, max_steps, bridge, n_threads)
    jac, jse = np.zeros((n, W)), np.zeros((n, W))
    nphi = {"poisson_fourier": 16, "poly1d": 2}.get(prob["problem"], 0)
    rec = np.zeros((n, int(n_paths), 4 + nphi)) if dump_paths else None
    steps = np.zeros((n, int(n_paths)), dtype=np.int32) if dump_paths else None
    rc = lib.orc_interface_jacobian(ctypes.byref(P), _ptr(nodes, ctypes.c_double), n,
                                    ctypes.byref(M), _ptr(jac, ctypes.c_double),
                                    _ptr(jse, ctypes.c_double), _ptr(rec, ctypes.c_double),
                                    _ptr(steps, ctypes.c_int32))
    if rc != 0:
        raise ValueError("oracle interface_jacobian: invalid arguments")
    if dump_paths:
        return jac, jse, rec, steps
    return jac, jse


def wos_solve(prob: dict, nodes, *, seed, n_paths, eps, max_steps=10**6, n_threads=None,
              dump_paths=False, node_ids=None):
    """Walk on Spheres for Eq. 1.1 (Sec. 2.1): mean, se, n per node, total
    steps, and with dump_paths per-path score[n, N], steps[n, N] and the
    projected stopping point exit[n, N, 2]."""
    lib = _load()
    nodes = np.ascontiguousarray(nodes, dtype=np.float64).reshape(-1, int(prob["dim"]))
    n = nodes.shape[0]
    P, keep = _problem(prob)
    M = _mc(seed, 1.0, n_paths, max_steps, False, n_threads)
    mean, se = np.zeros(n), np.zeros(n)
    cnt = np.zeros(n, dtype=np.int64)
    score = np.zeros((n, n_paths)) if dump_paths else None
    steps = np.zeros((n, n_paths), dtype=np.int32) if dump_paths else None
    exitp = np.zeros((n, n_paths, 2)) if dump_paths else None
    ids = None if node_ids is None else np.ascontiguousarray(node_ids, dtype=np.int64)
    ts = ctypes.c_int64(0)
    rc = lib.orc_wos_solve(ctypes.byref(P), _ptr(nodes, ctypes.c_double), n,
                           _ptr(ids, ctypes.c_int64), ctypes.byref(M), float(eps),
                           _ptr(mean, ctypes.c_double), _ptr(se, ctypes.c_double),
                           _ptr(cnt, ctypes.c_int64), _ptr(score, ctypes.c_double),
                           _ptr(steps, ctypes.c_int32), ctypes.byref(ts),
                           _ptr(exitp, ctypes.c_double))
    if rc != 0:
        raise ValueError("oracle wos_solve: invalid arguments")
    out = {"mean": mean, "se": se, "n": cnt, "total_steps": ts.value}
    if dump_paths:
        out["score"], out["steps"], out["exit"] = score, steps, exitp
    return out


def branching_solve(prob: dict, nodes_xt, *, seed, n_trees, max_particles=4096,
                    max_depth=64, n_threads=None, dump_trees=False):
    """Branching-diffusion estimate of u(x, t) for Eq. 3.1 / Sec. 3.2."""
    lib = _load()
    d = int(prob["dim"])
    nodes_xt = np.ascontiguousarray(nodes_xt, dtype=np.float64).reshape(-1, d + 1)
    n = nodes_xt.shape[0]
    P, keep = _problem(prob)
    M = _mc(seed, 1.0, n_trees, 1, False, n_threads)
    mean, se = np.zeros(n), np.zeros(n)
    kept = np.zeros(n, dtype=np.int64)
    disc = np.zeros(n, dtype=np.int64)
    ts = np.zeros((n, n_trees)) if dump_trees else None
    tg = np.zeros((n, n_trees), dtype=np.int32) if dump_trees else None
    rc = lib.orc_branching_solve(ctypes.byref(P), _ptr(nodes_xt, ctypes.c_double), n,
                                 ctypes.byref(M), int(max_particles), int(max_depth),
                                 _ptr(mean, ctypes.c_double), _ptr(se, ctypes.c_double),
                                 _ptr(kept, ctypes.c_int64), _ptr(disc, ctypes.c_int64),
                                 _ptr(ts, ctypes.c_double), _ptr(tg, ctypes.c_int32))
    if rc != 0:
        raise ValueError("oracle branching_solve: invalid arguments")
    out = {"mean": mean, "se": se, "n": kept, "discarded": disc}
    if dump_trees:
        out["score"], out["segments"] = ts, tg
    return out


def branching_grid_solve(prob: dict, nodes, times, *, seed, n_trees, dt=1e-3,
                         bridge=True, max_particles=4096, max_depth=64, n_threads=None,
                         dump_trees=False):
    """Branching estimate of u(x, T_i) for every time of the grid `times` from
    one tree per sample (Algorithm 3.1), in free space or with absorbing
    boundaries and boundary data g (Eq. 3.2).  mean/se are [n, m]."""
    lib = _load()
    d = int(prob["dim"])
    nodes = np.ascontiguousarray(nodes, dtype=np.float64).reshape(-1, d)
    times = np.ascontiguousarray(times, dtype=np.float64).ravel()
    n, m = nodes.shape[0], times.size
    P, keep = _problem(prob)
    M = _mc(seed, dt, n_trees, 1, bridge, n_threads)
    mean, se = np.zeros((n, m)), np.zeros((n, m))
    kept = np.zeros(n, dtype=np.int64)
    disc = np.zeros(n, dtype=np.int64)
    ts = np.zeros((n, n_trees, m)) if dump_trees else None
    tg = np.zeros((n, n_trees), dtype=np.int32) if dump_trees else None
    rc = lib.orc_branching_grid_solve(ctypes.byref(P), _ptr(nodes, ctypes.c_double), n,
                                      _ptr(times, ctypes.c_double), m, ctypes.byref(M),
                                      int(max_particles), int(max_depth),
                                      _ptr(mean, ctypes.c_double), _ptr(se, ctypes.c_double),
                                      _ptr(kept, ctypes.c_int64), _ptr(disc, ctypes.c_int64),
                                      _ptr(ts, ctypes.c_double), _ptr(tg, ctypes.c_int32))
    if rc != 0:
        raise ValueError("oracle branching_grid_solve: invalid arguments")
    out = {"mean": mean, "se": se, "n": kept, "discarded": disc}
    if dump_trees:
        out["score"], out["steps"] = ts, tg
    return out


def mlmc_level(prob: dict, nodes, *, seed, dt0, level, refine=2, n_paths, max_steps=10**8,
               bridge=True, n_threads=None, dump_paths=False):
    """One level of the multilevel estimator (Sec. 2.1): mean and variance per
    node of P_l - P_{l-1} (P_0 at level 0) from coupled fine/coarse Euler
    paths, plus the fine and coarse means."""
    lib = _load()
    d = int(prob["dim"])
    nodes = np.ascontiguousarray(nodes, dtype=np.float64).reshape(-1, d)
    n = nodes.shape[0]
    P, keep = _problem(prob)
    M = _mc(seed, dt0, n_paths, max_steps, bridge, n_threads)
    mean, var, fm, cm = np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(n)
    diff = np.zeros((n, n_paths)) if dump_paths else None
    steps = np.zeros((n, n_paths), dtype=np.int32) if dump_paths else None
    aux = np.zeros((n, n_paths, 8)) if dump_paths else None
    cap = ctypes.c_int64(0)
    rc = lib.orc_mlmc_level(ctypes.byref(P), _ptr(nodes, ctypes.c_double), n, ctypes.byref(M),
                            int(level), int(refine), _ptr(mean, ctypes.c_double),
                            _ptr(var, ctypes.c_double), _ptr(fm, ctypes.c_double),
                            _ptr(cm, ctypes.c_double), _ptr(diff, ctypes.c_double),
                            _ptr(steps, ctypes.c_int32), ctypes.byref(cap),
                            _ptr(aux, ctypes.c_double))
    if rc != 0:
        raise ValueError("oracle mlmc_level: invalid arguments")
    out = {"mean": mean, "var": var, "fine_mean": fm, "coarse_mean": cm, "capped": cap.value}
    if dump_paths:
        # aux per pair: fine score, coarse score, fine exit step, coarse exit
        # step (in coarse steps; negative: capped), fine and coarse exit points
        out["diff"], out["steps"], out["aux"] = diff, steps, aux
    return out


def mlmc_solve(prob: dict, nodes, *, seed, dt0, refine=2, n_per_level, bridge=True,
               n_threads=None):
    """Multilevel estimate: sum of the level means; se = sqrt(sum var_l / N_l)."""
    levels = [mlmc_level(prob, nodes, seed=seed, dt0=dt0, level=l, refine=refine, n_paths=N,
                         bridge=bridge, n_threads=n_threads)
              for l, N in enumerate(n_per_level)]
    mean = sum(L["mean"] for L in levels)
    se = np.sqrt(sum(L["var"] / N for L, N in zip(levels, n_per_level)))
    return {"mean": mean, "se": se, "levels": levels}


def grid_ticks_per_unit(t_max: float) -> float:
    """Integer time scale of the grid solver: 2^(31 - e) for t_max = f 2^e."""
    return _load().orc_grid_ticks_per_unit(float(t_max))


# --------------------------------------------------------------------------
# Deterministic stage (Sec. 2.1: interpolator and subdomain solver)
# --------------------------------------------------------------------------
def spline_interface(s_nodes, values, s_query, end0, end1, s0=0.0, s1=1.0):
    """Cubic spline with not-a-knot end conditions through (s0, end0),
    (s_k, values_k), (s1, end1), evaluated at s_query (the interpolator that
    turns nodal values into Dirichlet data on an interface, Sec. 2.1)."""
    from scipy.interpolate import CubicSpline
    s = np.concatenate([[s0], np.asarray(s_nodes, dtype=np.float64), [s1]])
    v = np.concatenate([[end0], np.asarray(values, dtype=np.float64), [end1]])
    return CubicSpline(s, v, bc_type="not-a-knot")(np.asarray(s_query, dtype=np.float64))


def stencil_solve(u_boundary: np.ndarray, h, sigma: float = 1.0) -> np.ndarray:
    """Exact solution of the 5-point (2-D) or 7-point (3-D) finite-difference
    Laplace system on a tensor grid: interior values satisfy
    sum_k (u[i+e_k] - 2 u[i] + u[i-e_k]) / h_k^2 = 0, boundary entries of
    `u_boundary` are Dirichlet data (the subdomain solver of Sec. 2.1 for the
    Laplace problem Eq. 1.1).  Direct sparse solve (SciPy), arrays indexed
    [z][y][x] / [y][x]."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    u = np.array(u_boundary, dtype=np.float64, copy=True)
    shape = u.shape
    dim = u.ndim
    h = np.broadcast_to(np.asarray(h, dtype=np.float64), (dim,))  # h per axis, x first
    interior = np.zeros(shape, dtype=bool)
    interior[tuple(slice(1, -1) for _ in range(dim))] = True
    idx = -np.ones(shape, dtype=np.int64)
    nint = int(interior.sum())
    idx[interior] = np.arange(nint)
    rows, cols, vals = [], [], []
    rhs = np.zeros(nint)
    pts = np.argwhere(interior)
    diag = 0.0
    for ax in range(dim):
        diag += 2.0 / h[dim - 1 - ax] ** 2
    for p in pts:
        r = idx[tuple(p)]
        rows.append(r); cols.append(r); vals.append(diag)
        for ax in range(dim):
            w = 1.0 / h[dim - 1 - ax] ** 2   # array axis ax <-> coordinate dim-1-ax
            for sgn in (-1, 1):
                q = p.copy(); q[ax] += sgn
                j = idx[tuple(q)]
                if j >= 0:
                    rows.append(r); cols.append(j); vals.append(-w)
                else:
                    rhs[r] += w * u[tuple(q)]
    A = sp.csr_matrix((vals, (rows, cols)), shape=(nint, nint))
    u[interior] = spla.spsolve(A, rhs)
    return u


def plane_boundary_points(axis: int, pos: float, n_bnd: int) -> np.ndarray:
    """Points on the perimeter of the internal plane x_axis = pos of the unit
    cube: n_bnd per edge (equispaced, corners included once), as 3-D points."""
    t = np.linspace(0.0, 1.0, n_bnd + 1)[:-1]
    s = np.concatenate([t, np.ones_like(t), 1.0 - t, np.zeros_like(t)])
    r = np.concatenate([np.zeros_like(t), t, np.ones_like(t), 1.0 - t])
    other = [a for a in range(3) if a != axis]
    pts = np.zeros((s.size, 3))
    pts[:, axis] = pos
    pts[:, other[0]] = s
    pts[:, other[1]] = r
    return pts


def plane_interface(prob: dict, axis: int, pos: float, nodes, values, query, n_bnd: int = 32):
    """Interface interpolation on an internal plane x_axis = pos of the unit
    cube (Sec. 2.1: the nodal values become Dirichlet data on the interface;
    Chebyshev or RBF interpolation are named there): a radial basis function
    interpolant with the cubic kernel |r|^3 and a linear polynomial term
    (SciPy's RBFInterpolator, a library routine) through the Monte Carlo
    nodes on the plane and n_bnd points per edge of the plane's perimeter,
    where the boundary data g are known, evaluated at the query points."""
    other = [a for a in range(3) if a != axis]
    nodes = np.asarray(nodes, dtype=np.float64)
    bnd = plane_boundary_points(axis, pos, n_bnd)
    gb = eval_coeffs_many(prob, bnd)[:, 5]
    pts = np.concatenate([nodes[:, other], bnd[:, other]])
    vals = np.concatenate([np.asarray(values, dtype=np.float64), gb])
    return rbf_interp(pts, vals, np.asarray(query, dtype=np.float64)[:, other])


def rbf_interp(points, values, query):
    """Cubic radial basis function interpolant |r|^3 with a linear polynomial
    term through (points, values), evaluated at query (SciPy's
    RBFInterpolator)."""
    from scipy.interpolate import RBFInterpolator
    return RBFInterpolator(np.asarray(points, dtype=np.float64),
                           np.asarray(values, dtype=np.float64), kernel="cubic",
                           degree=1)(np.asarray(query, dtype=np.float64))


def elliptic_box_solve(prob: dict, u_boundary: np.ndarray, lo, hi) -> np.ndarray:
    """Exact solution of the finite-difference system of the elliptic
    problem (1/2) sigma^2 Lap u + b . grad u + c u + f = 0 (Eq. 2.3 without
    time) on the box [lo, hi] with the tensor grid of u_boundary's shape
    ([n2][n1][n0], or [n1][n0] in 2-D), Dirichlet data in its boundary layer:
    7-point (5-point) second differences and central first differences,
    c and f at the grid point.  Direct sparse solve (SciPy)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    u = np.array(u_boundary, dtype=np.float64, copy=True)
    dim = u.ndim
    shape = u.shape                      # array axis k <-> coordinate dim - 1 - k
    h = [(hi[a] - lo[a]) / (shape[dim - 1 - a] - 1) for a in range(dim)]
    grids = [lo[a] + h[a] * np.arange(shape[dim - 1 - a]) for a in range(dim)]
    mesh = np.meshgrid(*[grids[dim - 1 - k] for k in range(dim)], indexing="ij")
    X = np.stack([mesh[dim - 1 - a] for a in range(dim)], -1)     # [..., dim], x first
    interior = np.zeros(shape, dtype=bool)
    interior[tuple(slice(1, -1) for _ in range(dim))] = True
    idx = -np.ones(shape, dtype=np.int64)
    nint = int(interior.sum())
    idx[interior] = np.arange(nint)
    coef = eval_coeffs_many(prob, X[interior])
    s2 = float(prob.get("sigma", 1.0)) ** 2
    rows = [np.arange(nint)]
    cols = [np.arange(nint)]
    diag = coef[:, 3].copy()
    for a in range(dim):
        diag -= s2 / h[a] ** 2
    vals = [diag]
    rhs = -coef[:, 4].copy()
    pts = np.argwhere(interior)
    for a in range(dim):
        k = dim - 1 - a                  # array axis of coordinate a
        for sgn in (-1, 1):
            w = 0.5 * s2 / h[a] ** 2 + sgn * coef[:, a] / (2.0 * h[a])
            q = pts.copy()
            q[:, k] += sgn
            j = idx[tuple(q.T)]
            inner = j >= 0
            rows.append(np.arange(nint)[inner])
            cols.append(j[inner])
            vals.append(w[inner])
            rhs[~inner] -= w[~inner] * u[tuple(q[~inner].T)]
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nint, nint))
    u[interior] = spla.spsolve(A, rhs)
    return u
