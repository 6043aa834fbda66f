"""Path-by-path comparison of a GPU solve with the FP64 oracle on shared
Philox streams (helper of the GPU parity tests; not a test module).

Both sides draw the same random numbers, so every path is the same random
path.  A binary32 path still rounds its position, so it can take an exit
decision at another step than the binary64 oracle (|U - P| or the distance to
the boundary below binary32 rounding), or leave through another face at the
same step (an exit near an edge or a corner).  Such paths are exit flips:
legitimate, counted and reported.  Every other path exits at the same step
through the same face, and its score must agree with the oracle's within the
per-path bound; the per-node means over those paths must agree to 1e-5
relative (the scope's node tolerance).

Exit faces are read off the exit points: a projected or crossing point has
one coordinate exactly on a face plane (0 or 1; 1/2 on the L-shape's notch).

Per-path bound for binary32 paths (path_bound).  Each Euler step rounds the
updated position once or twice (an FMA, an add) at 2^-24 relative, |X| <= 1,
so after n steps the exit point is off by at most ~2^-23 (n + 8) per
coordinate (the 8 covers the exit-point construction).  The score g(X_tau)
Y + Z then moves by at most |grad g| times that, plus a few binary32
roundings of the evaluation itself.  With G = |grad g| at the oracle's exit
point (Y <= 1 for these families):
    |s_gpu - s_oracle| <= 2^-22 ((n + 8) G + 16 (1 + |s|)) + G |x_gpu - x_oracle|,
twice the linear worst case, plus the measured distance of the two exit
points.  That last term covers a hard exit through the boundary at a grazing
angle: the crossing point X + t (X' - X) with t = (face - X_k)/(X'_k - X_k)
carries the rounding of X_k amplified by |X' - X| / |X'_k - X_k|.  Where the
exit points are more than 1e-3 apart (such a crossing, ill-conditioned) the
path counts as an exit flip, like a change of exit step or face.  Binary64
paths use a plain relative tolerance.
"""
from __future__ import annotations

import json
import os

import numpy as np

NODE_REL_TOL = 1e-5
EXIT_FLIP_DIST = 1e-3  # exit points farther apart than this at the same step and face


def exit_face(x: np.ndarray, geometry: str) -> np.ndarray:
    """Face code of exit points x [..., dim]: 3 * axis + (0 at 0, 1 at 1,
    2 at 1/2), for the first axis on a face plane; -1 for an interior point."""
    x = np.asarray(x, dtype=np.float64)
    code = np.full(x.shape[:-1], -1, dtype=np.int64)
    planes = (0.0, 1.0, 0.5) if geometry == "l_shape" else (0.0, 1.0)
    for axis in reversed(range(x.shape[-1])):
        for k, v in enumerate(planes):
            code = np.where(x[..., axis] == v, 3 * axis + k, code)
    return code


def grad_norm(prob: dict, x: np.ndarray) -> np.ndarray:
    """|grad g| of the family's boundary data at points x [..., dim]."""
    x = np.asarray(x, dtype=np.float64)
    kind = prob["problem"]
    if kind == "laplace_expcos":                     # g = e^x cos y
        return np.exp(x[..., 0])
    if kind == "elliptic_manufactured":              # g = sin(pi x) sin(pi y) e^z
        sx, cx = np.sin(np.pi * x[..., 0]), np.cos(np.pi * x[..., 0])
        sy, cy = np.sin(np.pi * x[..., 1]), np.cos(np.pi * x[..., 1])
        return np.exp(x[..., 2]) * np.sqrt((np.pi * cx * sy) ** 2 + (np.pi * sx * cy) ** 2
                                           + (sx * sy) ** 2)
    if kind == "poisson_fourier":                    # g = sum theta_mn cos(m pi x) cos(n pi y)
        th = np.asarray(prob["params"][:64]).reshape(8, 8)
        m = np.arange(8) * np.pi
        cxm, sxm = np.cos(x[..., 0, None] * m), np.sin(x[..., 0, None] * m)
        cyn, syn = np.cos(x[..., 1, None] * m), np.sin(x[..., 1, None] * m)
        gx = np.einsum("...m,mn,...n->...", -m * sxm, th, cyn)
        gy = np.einsum("...m,mn,...n->...", cxm, th, -m * syn)
        return np.hypot(gx, gy)
    raise ValueError(kind)


def path_bound(prob: dict, o: dict) -> np.ndarray:
    """Per-path bound on |s_gpu - s_oracle| for binary32 paths that exit at
    the same step through the same face (see the module docstring)."""
    n = np.abs(np.asarray(o["steps"], dtype=np.float64))
    G = grad_norm(prob, o["exit"])
    return 2.0 ** -22 * ((n + 8.0) * G + 16.0 * (1.0 + np.abs(o["score"])))


def compare_paths(g: dict, o: dict, *, path_tol=None, geometry: str | None = None,
                  prob: dict | None = None) -> dict:
    """Classify every (node, path): exit-step flips, exit-face flips (same
    step, other face), and paths with the same exit; among the latter, count
    score mismatches beyond the per-path bound (path_bound(prob, o) when prob
    is given, else path_tol * max(1, |s|)) and form the per-node relative
    difference of the means."""
    sg = np.asarray(g["score"].cpu().numpy() if hasattr(g["score"], "cpu") else g["score"])
    stg = np.asarray(g["steps"].cpu().numpy() if hasattr(g["steps"], "cpu") else g["steps"])
    so, sto = np.asarray(o["score"]), np.asarray(o["steps"])
    step_flip = stg != sto
    dx = np.zeros(so.shape)
    if geometry is not None and "exit" in g and "exit" in o:
        xg = g["exit"].cpu().numpy() if hasattr(g["exit"], "cpu") else np.asarray(g["exit"])
        face_flip = ~step_flip & (exit_face(xg, geometry) != exit_face(o["exit"], geometry))
        dx = np.abs(xg - o["exit"]).max(-1)
        face_flip |= ~step_flip & (dx > EXIT_FLIP_DIST)
    else:
        face_flip = np.zeros_like(step_flip)
    same = ~(step_flip | face_flip)
    scale = np.maximum(1.0, np.abs(so))
    prel = np.where(same, np.abs(sg - so) / scale, 0.0)
    if prob is not None:
        bound = path_bound(prob, o) + grad_norm(prob, o["exit"]) * dx
    else:
        bound = path_tol * scale
    ratio = np.where(same, np.abs(sg - so) / bound, 0.0)
    mismatch = same & (ratio > 1.0)
    cnt = same.sum(1)
    mg = np.where(same, sg, 0.0).sum(1) / np.maximum(cnt, 1)
    mo = np.where(same, so, 0.0).sum(1) / np.maximum(cnt, 1)
    nscale = np.maximum(np.abs(mo), 0.1 * np.sqrt((so ** 2).mean(1)))
    node_rel = np.abs(mg - mo) / nscale
    total = step_flip.size
    return {
        "paths": int(total),
        "step_flips": int(step_flip.sum()),
        "face_flips": int(face_flip.sum()),
        "flip_frac": float((step_flip | face_flip).sum() / max(total, 1)),
        "mismatch": int(mismatch.sum()),
        "max_path_rel": float(prel.max()) if total else 0.0,
        "max_bound_ratio": float(ratio.max()) if total else 0.0,
        "max_exit_dist": float(np.where(same, dx, 0.0).max()) if total else 0.0,
        "node_rel_max": float(node_rel.max()) if node_rel.size else 0.0,
        "min_same": int(cnt.min()) if cnt.size else 0,
        "node_rel": node_rel,
        "same": same,
    }


def report(name: str, st: dict) -> str:
    """One line for the test log; with PDD_PARITY_LOG set, also appended to
    that file as JSON (the measured flip fractions are recorded from it)."""
    keys = ("paths", "step_flips", "face_flips", "flip_frac", "mismatch", "max_path_rel",
            "max_bound_ratio", "max_exit_dist", "node_rel_max", "min_same")
    rec = {"case": name, **{k: st[k] for k in keys}}
    path = os.environ.get("PDD_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(rec) + "\n")
    line = (f"[parity] {name}: flips {st['flip_frac']:.2e} ({st['step_flips']} step, "
            f"{st['face_flips']} face or place of {st['paths']}), mismatches {st['mismatch']}, "
            f"max path rel {st['max_path_rel']:.2e} ({st['max_bound_ratio']:.2f} of the bound), "
            f"max node rel {st['node_rel_max']:.2e}")
    print(line)
    return line


def check(name: str, st: dict, *, flip_max: float, node_tol: float = NODE_REL_TOL) -> None:
    """The parity bar: no same-exit path outside the per-path bound, exit
    flips within flip_max, per-node means within node_tol."""
    report(name, st)
    assert st["mismatch"] == 0, (name, st["mismatch"], st["max_path_rel"])
    assert st["flip_frac"] <= flip_max, (name, st["flip_frac"], flip_max)
    assert st["min_same"] > 0, name
    assert st["node_rel_max"] <= node_tol, (name, st["node_rel_max"])
