"""Python face of the C ABI: the same operations as include/pdd.h, with torch
tensors for device memory and torch's current CUDA stream.  Every step of the
method runs in libpdd.so; this module only checks types and marshals pointers.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib

_F64, _I64, _I32, _U32 = torch.float64, torch.int64, torch.int32, torch.uint32


def _stream_handle(device: torch.device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _dev_f64(t, device, shape_last=None) -> torch.Tensor:
    t = torch.as_tensor(t, dtype=_F64)
    if t.device != device:
        t = t.to(device, non_blocking=True)
    return t.contiguous()


class Context:
    """A library context for one problem (a dict from ``workloads``)."""

    def __init__(self, prob: dict, device: int | torch.device = 0):
        self.lib = _lib.load()
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        self.prob = prob
        params = np.ascontiguousarray(prob.get("params", np.zeros(0)), dtype=np.float64)
        self._params = params
        p = _lib.Problem(_lib.PROBLEM[prob["problem"]], _lib.GEOMETRY[prob["geometry"]],
                         int(prob["dim"]), int(params.size),
                         params.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         float(prob.get("sigma", 1.0)))
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = self.lib.pdd_create(ctypes.byref(h), ctypes.byref(p), self.device.index,
                                     _stream_handle(self.device))
        _lib.check(st, create=True)
        self.handle = h

    # ------------------------------------------------------------------
    def close(self):
        if getattr(self, "handle", None):
            self.lib.pdd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _bind_stream(self):
        _lib.check(self.lib.pdd_set_stream(self.handle, _stream_handle(self.device)), self.handle)

    def set_tuning(self, blocks_per_sm: int = 0, wave_max_paths: int = 0):
        """pdd_set_tuning: launch shape / wave size (results unchanged)."""
        _lib.check(self.lib.pdd_set_tuning(self.handle, int(blocks_per_sm), int(wave_max_paths)),
                   self.handle)

    def profile(self, enable: bool = True):
        """pdd_profile: time every path-kernel launch with CUDA events."""
        _lib.check(self.lib.pdd_profile(self.handle, int(bool(enable))), self.handle)

    def profile_read(self):
        """pdd_profile_read: (summed kernel ms, launches) since the last read."""
        ms, n = ctypes.c_double(0.0), ctypes.c_int64(0)
        with torch.cuda.device(self.device):
            _lib.check(self.lib.pdd_profile_read(self.handle, ctypes.byref(ms), ctypes.byref(n)),
                       self.handle)
        return ms.value, n.value

    # ------------------------------------------------------------------
    def interface_solve(self, nodes, *, seed: int, dt: float, n_paths: int,
                        max_steps: int = 2**31 - 1, precision: str = "fp32",
                        bridge: bool = True, path_offset: int = 0, node_offset: int = 0,
                        dump_paths: bool = False, diag: bool = False, out=None) -> dict:
        """pdd_interface_solve on torch tensors.

        nodes: [n, dim] float64 (CUDA tensor, or a CPU tensor that is copied).
        node_offset: stream index of the first node (a node block of a larger
        list draws that list's streams).
        Returns mean, se (float64 [n]) and n (int64 [n]) as CUDA tensors; with
        diag or dump_paths also path_steps / capped (host ints) and flags
        (int32 [n], PDD_NODE_* bits) and, with dump_paths, score [n, n_paths]
        float64, steps [n, n_paths] int32 and exit [n, n_paths, dim] float64."""
        dim = int(self.prob["dim"])
        nodes = _dev_f64(nodes, self.device).reshape(-1, dim)
        n = nodes.shape[0]
        if out is None:
            mean = torch.empty(n, dtype=_F64, device=self.device)
            se = torch.empty(n, dtype=_F64, device=self.device)
            npaths = torch.empty(n, dtype=_I64, device=self.device)
        else:
            mean, se, npaths = out
        mc = _lib.MCParams(int(seed) & (2**64 - 1), float(dt), int(n_paths), int(max_steps),
                           int(path_offset), _lib.PRECISION[precision], int(bool(bridge)),
                           int(node_offset))
        res = {"mean": mean, "se": se, "n": npaths}
        dg = None
        if diag or dump_paths:
            dg = _lib.Diag()
            res["flags"] = torch.zeros(n, dtype=_I32, device=self.device)
            dg.d_node_flags = res["flags"].data_ptr()
            if dump_paths:
                res["score"] = torch.empty((n, int(n_paths)), dtype=_F64, device=self.device)
                res["steps"] = torch.empty((n, int(n_paths)), dtype=_I32, device=self.device)
                res["exit"] = torch.empty((n, int(n_paths), dim), dtype=_F64, device=self.device)
                dg.d_path_score = res["score"].data_ptr()
                dg.d_path_steps = res["steps"].data_ptr()
                dg.d_path_exit = res["exit"].data_ptr()
        with torch.cuda.device(self.device):
            self._bind_stream()
            st = self.lib.pdd_interface_solve(self.handle, nodes.data_ptr(), n, ctypes.byref(mc),
                                              mean.data_ptr(), se.data_ptr(), npaths.data_ptr(),
                                              ctypes.byref(dg) if dg is not None else None)
        res["status"] = _lib.check(st, self.handle, allow=(_lib.PDD_OK, _lib.PDD_ECAP))
        if dg is not None:
            res["path_steps"], res["capped"] = int(dg.path_steps), int(dg.capped)
        return res

    def branching_solve(self, nodes_xt, *, seed: int, n_trees: int, max_particles: int = 4096,
                        max_depth: int = 64, tree_offset: int = 0, dump_trees: bool = False,
                        diag: bool = False, out=None) -> dict:
        """pdd_branching_solve: nodes_xt [n, dim+1] float64 (position, then t).

        Returns mean, se, n (trees kept); with diag/dump_trees also segments
        (total) and discarded (host ints) and flags (int32 [n], PDD_NODE_*);
        with dump_trees score [n, n_trees] (NaN = discarded) and segs
        [n, n_trees] (negative = discarded)."""
        dim = int(self.prob["dim"])
        nodes_xt = _dev_f64(nodes_xt, self.device).reshape(-1, dim + 1)
        n = nodes_xt.shape[0]
        if out is None:
            mean = torch.empty(n, dtype=_F64, device=self.device)
            se = torch.empty(n, dtype=_F64, device=self.device)
            kept = torch.empty(n, dtype=_I64, device=self.device)
        else:
            mean, se, kept = out
        bp = _lib.BranchParams(int(seed) & (2**64 - 1), int(n_trees), int(tree_offset),
                               int(max_particles), int(max_depth), 0)
        res = {"mean": mean, "se": se, "n": kept}
        dg = None
        if diag or dump_trees:
            dg = _lib.Diag()
            res["flags"] = torch.zeros(n, dtype=_I32, device=self.device)
            dg.d_node_flags = res["flags"].data_ptr()
            if dump_trees:
                res["score"] = torch.empty((n, int(n_trees)), dtype=_F64, device=self.device)
                res["segs"] = torch.empty((n, int(n_trees)), dtype=_I32, device=self.device)
                dg.d_path_score = res["score"].data_ptr()
                dg.d_path_steps = res["segs"].data_ptr()
        with torch.cuda.device(self.device):
            self._bind_stream()
            st = self.lib.pdd_branching_solve(self.handle, nodes_xt.data_ptr(), n, ctypes.byref(bp),
                                              mean.data_ptr(), se.data_ptr(), kept.data_ptr(),
                                              ctypes.byref(dg) if dg is not None else None)
        res["status"] = _lib.check(st, self.handle, allow=(_lib.PDD_OK, _lib.PDD_ECAP))
        if dg is not None:
            res["segments"], res["discarded"] = int(dg.path_steps), int(dg.capped)
        return res

    def branching_grid_solve(self, nodes, times, *, seed: int, n_trees: int, dt: float = 1e-3,
                             bridge: bool = True, max_particles: int = 4096, max_depth: int = 64,
                             tree_offset: int = 0, dump_trees: bool = False,
                             diag: bool = False) -> dict:
        """pdd_branching_grid_solve: nodes [n, dim] float64, times [m] (host).

        Returns mean [n, m], se [n, m], n (trees kept) [n]; with diag/dump_trees
        also steps (total) and discarded (host ints); with dump_trees score
        [n, n_trees, m] (NaN = discarded) and tree_steps [n, n_trees]."""
        dim = int(self.prob["dim"])
        nodes = _dev_f64(nodes, self.device).reshape(-1, dim)
        n = nodes.shape[0]
        tm = np.ascontiguousarray(np.asarray(times, dtype=np.float64).ravel())
        m = int(tm.size)
        mean = torch.empty((n, m), dtype=_F64, device=self.device)
        se = torch.empty((n, m), dtype=_F64, device=self.device)
        kept = torch.empty(n, dtype=_I64, device=self.device)
        bp = _lib.GridBranchParams(int(seed) & (2**64 - 1), int(n_trees), int(tree_offset),
                                   int(max_particles), int(max_depth), int(bool(bridge)), float(dt))
        res = {"mean": mean, "se": se, "n": kept}
        dg = None
        if diag or dump_trees:
            dg = _lib.Diag()
            if dump_trees:
                res["score"] = torch.empty((n, int(n_trees), m), dtype=_F64, device=self.device)
                res["tree_steps"] = torch.empty((n, int(n_trees)), dtype=_I32, device=self.device)
                dg.d_path_score = res["score"].data_ptr()
                dg.d_path_steps = res["tree_steps"].data_ptr()
        with torch.cuda.device(self.device):
            self._bind_stream()
            st = self.lib.pdd_branching_grid_solve(
                self.handle, nodes.data_ptr(), n, tm.ctypes.data, m, ctypes.byref(bp),
                mean.data_ptr(), se.data_ptr(), kept.data_ptr(),
                ctypes.byref(dg) if dg is not None else None)
        res["status"] = _lib.check(st, self.handle, allow=(_lib.PDD_OK, _lib.PDD_ECAP))
        if dg is not None:
            res["steps"], res["discarded"] = int(dg.path_steps), int(dg.capped)
        return res

    def mlmc_level(self, nodes, *, seed: int, dt0: float, level: int, n_paths: int,
                   refine: int = 2, max_steps: int = 2**31 - 1, precision: str = "fp32",
                   bridge: bool = True, dump_paths: bool = False, diag: bool = False) -> dict:
        """pdd_mlmc_level: mean/var of P_l - P_{l-1} per node, fine and coarse means."""
        nodes = _dev_f64(nodes, self.device).reshape(-1, int(self.prob["dim"]))
        n = nodes.shape[0]
        res = {k: torch.empty(n, dtype=_F64, device=self.device)
               for k in ("mean", "var", "fine_mean", "coarse_mean")}
        mp = _lib.MlmcParams(int(seed) & (2**64 - 1), int(n_paths), int(max_steps), float(dt0),
                             int(level), int(refine), _lib.PRECISION[precision], int(bool(bridge)))
        dg = None
        if diag or dump_paths:
            dg = _lib.Diag()
            if dump_paths:
                res["diff"] = torch.empty((n, int(n_paths)), dtype=_F64, device=self.device)
                res["steps"] = torch.empty((n, int(n_paths)), dtype=_I32, device=self.device)
                res["aux"] = torch.empty((n, int(n_paths), 8), dtype=_F64, device=self.device)
                dg.d_path_score = res["diff"].data_ptr()
                dg.d_path_steps = res["steps"].data_ptr()
                dg.d_path_aux = res["aux"].data_ptr()
        with torch.cuda.device(self.device):
            self._bind_stream()
            st = self.lib.pdd_mlmc_level(self.handle, nodes.data_ptr(), n, ctypes.byref(mp),
                                         res["mean"].data_ptr(), res["var"].data_ptr(),
                                         res["fine_mean"].data_ptr(), res["coarse_mean"].data_ptr(),
                                         ctypes.byref(dg) if dg is not None else None)
        res["status"] = _lib.check(st, self.handle, allow=(_lib.PDD_OK, _lib.PDD_ECAP))
        if dg is not None:
            res["path_steps"], res["capped"] = int(dg.path_steps), int(dg.capped)
        return res

    def mlmc_solve(self, nodes, *, seed: int, dt0: float, n_per_level, refine: int = 2,
                   max_steps: int = 2**31 - 1, precision: str = "fp32", bridge: bool = True,
                   diag: bool = False) -> dict:
        """pdd_mlmc_solve: the multilevel estimate (levels summed on the device).
        Returns mean, se [n] and levels (per level: mean, var [n])."""
        nodes = _dev_f64(nodes, self.device).reshape(-1, int(self.prob["dim"]))
        n = nodes.shape[0]
        L = len(n_per_level)
        counts = (ctypes.c_int64 * L)(*[int(N) for N in n_per_level])
        mean = torch.empty(n, dtype=_F64, device=self.device)
        se = torch.empty(n, dtype=_F64, device=self.device)
        lmean = torch.empty((L, n), dtype=_F64, device=self.device)
        lvar = torch.empty((L, n), dtype=_F64, device=self.device)
        mp = _lib.MlmcParams(int(seed) & (2**64 - 1), 0, int(max_steps), float(dt0), 0,
                             int(refine), _lib.PRECISION[precision], int(bool(bridge)))
        dg = _lib.Diag() if diag else None
        with torch.cuda.device(self.device):
            self._bind_stream()
            st = self.lib.pdd_mlmc_solve(self.handle, nodes.data_ptr(), n, ctypes.byref(mp), L,
                                         counts, mean.data_ptr(), se.data_ptr(),
                                         lmean.data_ptr(), lvar.data_ptr(),
                                         ctypes.byref(dg) if dg is not None else None)
        res = {"mean": mean, "se": se,
               "levels": [{"mean": lmean[l], "var": lvar[l]} for l in range(L)],
               "status": _lib.check(st, self.handle, allow=(_lib.PDD_OK, _lib.PDD_ECAP))}
        if dg is not None:
            res["path_steps"], res["capped"] = int(dg.path_steps), int(dg.capped)
        return res

    def subdomain_solve(self, lo, hi, n, iface_axis: int, iface_side: int, iface_s, iface_vals,
                        *, method: str = "cg", max_iter: int = 100000, tol: float = 1e-12,
                        out=None) -> dict:
        """pdd_subdomain_solve on a 2-D box: returns u [n[1], n[0]] (CUDA), iters, resid."""
        s = _dev_f64(iface_s, self.device).reshape(-1)
        v = _dev_f64(iface_vals, self.device).reshape(-1)
        nx, ny = int(n[0]), int(n[1])
        u = out if out is not None else torch.empty((ny, nx), dtype=_F64, device=self.device)
        sd = _lib.Subdomain((ctypes.c_double * 3)(lo[0], lo[1], 0.0),
                            (ctypes.c_double * 3)(hi[0], hi[1], 0.0),
                            (ctypes.c_int32 * 3)(nx, ny, 1), int(iface_axis), int(iface_side),
                            _lib.STENCIL[method], int(max_iter), float(tol))
        it, res = ctypes.c_int64(0), ctypes.c_double(0.0)
        with torch.cuda.device(self.device):
            self._bind_stream()
            st = self.lib.pdd_subdomain_solve(self.handle, ctypes.byref(sd), s.data_ptr(),
                                              v.data_ptr(), s.numel(), u.data_ptr(),
                                              ctypes.byref(it), ctypes.byref(res))
        status = _lib.check(st, self.handle, allow=(_lib.PDD_OK, _lib.PDD_ETIMEOUT))
        return {"u": u, "iters": it.value, "resid": res.value, "status": status}

    def subdomain_solve3d(self, lo, hi, n, faces: dict, *, method: str = "dst",
                          max_iter: int = 200, tol: float = 1e-12, out=None) -> dict:
        """pdd_subdomain_solve on a 3-D box: faces maps a face index (2 axis +
        side) to its Dirichlet data (the face's full grid, the higher axis
        slow); the other faces take g.  Returns u [n2, n1, n0] (CUDA), iters,
        resid."""
        n0, n1, n2 = (int(v) for v in n)
        mask = 0
        parts = []
        for fc in sorted(faces):
            mask |= 1 << int(fc)
            parts.append(_dev_f64(faces[fc], self.device).reshape(-1))
        vals = torch.cat(parts) if parts else torch.zeros(0, dtype=_F64, device=self.device)
        u = out if out is not None else torch.empty((n2, n1, n0), dtype=_F64, device=self.device)
        sd = _lib.Subdomain((ctypes.c_double * 3)(*[float(v) for v in lo]),
                            (ctypes.c_double * 3)(*[float(v) for v in hi]),
                            (ctypes.c_int32 * 3)(n0, n1, n2), mask, 0, _lib.STENCIL[method],
                            int(max_iter), float(tol))
        it, res = ctypes.c_int64(0), ctypes.c_double(0.0)
        with torch.cuda.device(self.device):
            self._bind_stream()
            st = self.lib.pdd_subdomain_solve(self.handle, ctypes.byref(sd), None,
                                              vals.data_ptr() if vals.numel() else None,
                                              vals.numel(), u.data_ptr(), ctypes.byref(it),
                                              ctypes.byref(res))
        status = _lib.check(st, self.handle, allow=(_lib.PDD_OK, _lib.PDD_ETIMEOUT))
        return {"u": u, "iters": it.value, "resid": res.value, "status": status}

    def subdomain_solve3d_batch(self, boxes, n, *, method: str = "dst", max_iter: int = 200,
                                tol: float = 1e-12, out=None) -> dict:
        """pdd_subdomain_solve_batch: boxes is a list of (lo, hi, faces) with
        faces as for subdomain_solve3d, all on the same n = (n0, n1, n2) grid.
        Returns u [n_boxes, n2, n1, n0] (CUDA), the largest iters and resid,
        and each box's (iters_each, resid_each)."""
        n0, n1, n2 = (int(v) for v in n)
        nb = len(boxes)
        sds = (_lib.Subdomain * nb)()
        parts = []
        for b, (lo, hi, faces) in enumerate(boxes):
            mask = 0
            for fc in sorted(faces):
                mask |= 1 << int(fc)
                parts.append(_dev_f64(faces[fc], self.device).reshape(-1))
            sds[b] = _lib.Subdomain((ctypes.c_double * 3)(*[float(v) for v in lo]),
                                    (ctypes.c_double * 3)(*[float(v) for v in hi]),
                                    (ctypes.c_int32 * 3)(n0, n1, n2), mask, 0,
                                    _lib.STENCIL[method], int(max_iter), float(tol))
        vals = torch.cat(parts) if parts else torch.zeros(0, dtype=_F64, device=self.device)
        u = out if out is not None else torch.empty((nb, n2, n1, n0), dtype=_F64,
                                                    device=self.device)
        it, res = ctypes.c_int64(0), ctypes.c_double(0.0)
        it_each = (ctypes.c_int64 * nb)()
        res_each = (ctypes.c_double * nb)()
        with torch.cuda.device(self.device):
            self._bind_stream()
            st = self.lib.pdd_subdomain_solve_batch(self.handle, sds, nb,
                                                    vals.data_ptr() if vals.numel() else None,
                                                    vals.numel(), u.data_ptr(), ctypes.byref(it),
                                                    ctypes.byref(res), it_each, res_each)
        status = _lib.check(st, self.handle, allow=(_lib.PDD_OK, _lib.PDD_ETIMEOUT))
        return {"u": u, "iters": it.value, "resid": res.value, "status": status,
                "iters_each": list(it_each), "resid_each": list(res_each)}

    def interface_interp(self, planes, queries, *, n_bnd: int = 32) -> list:
        """pdd_interface_interp: planes is a list of (axis, pos, nodes [m, 3],
        values [m]); queries a list of [q, 3] point sets, one per plane.
        Returns the interpolated values per plane (CUDA tensors)."""
        P = len(planes)
        axis = (ctypes.c_int32 * P)(*[int(p[0]) for p in planes])
        pos = (ctypes.c_double * P)(*[float(p[1]) for p in planes])
        nodes = [_dev_f64(p[2], self.device).reshape(-1, 3) for p in planes]
        vals = [_dev_f64(p[3], self.device).reshape(-1) for p in planes]
        qs = [_dev_f64(q, self.device).reshape(-1, 3) for q in queries]
        cnt = (ctypes.c_int64 * P)(*[int(x.shape[0]) for x in nodes])
        qcnt = (ctypes.c_int64 * P)(*[int(q.shape[0]) for q in qs])
        d_nodes, d_vals, d_q = torch.cat(nodes), torch.cat(vals), torch.cat(qs)
        out = torch.empty(d_q.shape[0], dtype=_F64, device=self.device)
        with torch.cuda.device(self.device):
            self._bind_stream()
            st = self.lib.pdd_interface_interp(self.handle, P, axis, pos, cnt, d_nodes.data_ptr(),
                                               d_vals.data_ptr(), int(n_bnd), qcnt,
                                               d_q.data_ptr(), out.data_ptr())
        _lib.check(st, self.handle)
        return list(torch.split(out, [int(q.shape[0]) for q in qs]))

    def set_params(self, params):
        """pdd_set_params: new parameter values for the same family."""
        arr = np.ascontiguousarray(params, dtype=np.float64).reshape(-1)
        _lib.check(self.lib.pdd_set_params(self.handle,
                                           arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           int(arr.size)), self.handle)
        self._params = arr
        self.prob = dict(self.prob, params=arr)

    def interface_grad(self, nodes, *, seed: int, dt: float, n_paths: int, grad_out=None,
                       jacobian: bool = True, max_steps: int = 2**31 - 1, bridge: bool = True,
                       path_offset: int = 0, dump_paths: bool = False, diag: bool = False) -> dict:
        """pdd_interface_grad: jac/jac_se [n, 80] and, with grad_out [n], dtheta [64]
        and dphi [16] (all float64 CUDA tensors)."""
        dim = int(self.prob["dim"])
        nodes = _dev_f64(nodes, self.device).reshape(-1, dim)
        n = nodes.shape[0]
        res = {}
        jac = jse = gout = dth = dph = None
        if jacobian:
            jac = res["jac"] = torch.empty((n, 80), dtype=_F64, device=self.device)
            jse = res["jac_se"] = torch.empty((n, 80), dtype=_F64, device=self.device)
        if grad_out is not None:
            gout = _dev_f64(grad_out, self.device).reshape(-1)
            if gout.numel() != n:
                raise ValueError("grad_out must have one entry per node")
            dth = res["dtheta"] = torch.empty(64, dtype=_F64, device=self.device)
            dph = res["dphi"] = torch.empty(16, dtype=_F64, device=self.device)
        mc = _lib.MCParams(int(seed) & (2**64 - 1), float(dt), int(n_paths), int(max_steps),
                           int(path_offset), _lib.PRECISION["fp32"], int(bool(bridge)))
        dg = None
        if diag or dump_paths:
            dg = _lib.Diag()
            if dump_paths:
                res["score"] = torch.empty((n, int(n_paths)), dtype=_F64, device=self.device)
                res["steps"] = torch.empty((n, int(n_paths)), dtype=_I32, device=self.device)
                res["aux"] = torch.empty((n, int(n_paths), 18), dtype=_F64, device=self.device)
                dg.d_path_score = res["score"].data_ptr()
                dg.d_path_steps = res["steps"].data_ptr()
                dg.d_path_aux = res["aux"].data_ptr()
        ptr = lambda t: t.data_ptr() if t is not None else None
        with torch.cuda.device(self.device):
            self._bind_stream()
            st = self.lib.pdd_interface_grad(self.handle, nodes.data_ptr(), n, ctypes.byref(mc),
                                             ptr(gout), ptr(jac), ptr(jse), ptr(dth), ptr(dph),
                                             ctypes.byref(dg) if dg is not None else None)
        res["status"] = _lib.check(st, self.handle, allow=(_lib.PDD_OK, _lib.PDD_ECAP))
        if dg is not None:
            res["path_steps"], res["capped"] = int(dg.path_steps), int(dg.capped)
        return res

    def batch_solve(self, problems, nodes, problem_index, dt, *, seed: int, n_pilot: int,
                    n_min: int, n_max: int, target_se: float, max_steps: int = 2**31 - 1,
                    chunk: int = 0, bridge: bool = True, use_graph: bool = False,
                    diag: bool = False, out=None) -> dict:
        """pdd_batch_solve: problems is a list of workload dicts; nodes [n, 3]
        float64, problem_index [n] int32, dt [n] float64 (CUDA or CPU tensors)."""
        probs = []
        keep = []
        for pr in problems:
            prm = np.ascontiguousarray(pr.get("params", np.zeros(0)), dtype=np.float64)
            buf = prm if prm.size else np.zeros(1)
            keep.append(buf)
            probs.append(_lib.Problem(_lib.PROBLEM[pr["problem"]], _lib.GEOMETRY[pr["geometry"]],
                                      int(pr["dim"]), int(prm.size),
                                      buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      float(pr.get("sigma", 1.0))))
        arr = (_lib.Problem * len(probs))(*probs)
        nodes = _dev_f64(nodes, self.device).reshape(-1, 3)
        pidx = torch.as_tensor(problem_index, dtype=torch.int32).to(self.device).contiguous()
        dts = _dev_f64(dt, self.device).reshape(-1)
        n = nodes.shape[0]
        if out is None:
            mean = torch.empty(n, dtype=_F64, device=self.device)
            se = torch.empty(n, dtype=_F64, device=self.device)
            cnt = torch.empty(n, dtype=_I64, device=self.device)
        else:
            mean, se, cnt = out
        bn = _lib.BatchNodes(nodes.data_ptr(), pidx.data_ptr(), dts.data_ptr(), n)
        bp = _lib.BatchParams(int(seed) & (2**64 - 1), int(n_pilot), int(n_min), int(n_max),
                              float(target_se), int(max_steps), int(chunk), int(bool(bridge)))
        dg = _lib.Diag() if diag else None
        flags = None
        if dg is not None:
            flags = torch.zeros(n, dtype=_I32, device=self.device)
            dg.d_node_flags = flags.data_ptr()
        with torch.cuda.device(self.device):
            self._bind_stream()
            st = self.lib.pdd_batch_solve(self.handle, arr, len(probs), ctypes.byref(bn),
                                          ctypes.byref(bp), mean.data_ptr(), se.data_ptr(),
                                          cnt.data_ptr(), int(bool(use_graph)),
                                          ctypes.byref(dg) if dg is not None else None)
        res = {"mean": mean, "se": se, "n": cnt,
               "status": _lib.check(st, self.handle, allow=(_lib.PDD_OK, _lib.PDD_ECAP)),
               "_keep": (nodes, pidx, dts)}
        if dg is not None:
            res["path_steps"], res["capped"] = int(dg.path_steps), int(dg.capped)
            res["flags"] = flags
        return res

    def interface_solve_naive(self, nodes, *, seed: int, dt: float, n_paths: int,
                              max_steps: int = 2**31 - 1, bridge: bool = True, out=None) -> dict:
        """pdd_interface_solve_naive (one launch per node, thread per path)."""
        dim = int(self.prob["dim"])
        nodes = _dev_f64(nodes, self.device).reshape(-1, dim)
        n = nodes.shape[0]
        if out is None:
            out = (torch.empty(n, dtype=_F64, device=self.device),
                   torch.empty(n, dtype=_F64, device=self.device),
                   torch.empty(n, dtype=_I64, device=self.device))
        mc = _lib.MCParams(int(seed) & (2**64 - 1), float(dt), int(n_paths), int(max_steps), 0,
                           _lib.PRECISION["fp32"], int(bool(bridge)))
        with torch.cuda.device(self.device):
            self._bind_stream()
            st = self.lib.pdd_interface_solve_naive(self.handle, nodes.data_ptr(), n,
                                                    ctypes.byref(mc), out[0].data_ptr(),
                                                    out[1].data_ptr(), out[2].data_ptr())
        _lib.check(st, self.handle)
        return {"mean": out[0], "se": out[1], "n": out[2]}

    def autotune(self, nodes, *, seed: int, dt: float, n_paths: int, precision: str = "fp32",
                 bridge: bool = True, repeats: int = 2) -> dict:
        """pdd_autotune: pick the resident blocks per SM of the path kernels."""
        dim = int(self.prob["dim"])
        nodes = _dev_f64(nodes, self.device).reshape(-1, dim)
        n = nodes.shape[0]
        scratch = torch.empty(2 * n, dtype=_F64, device=self.device)
        mc = _lib.MCParams(int(seed) & (2**64 - 1), float(dt), int(n_paths), 2**31 - 1, 0,
                           _lib.PRECISION[precision], int(bool(bridge)))
        b, ms = ctypes.c_int32(0), ctypes.c_double(0.0)
        with torch.cuda.device(self.device):
            self._bind_stream()
            st = self.lib.pdd_autotune(self.handle, nodes.data_ptr(), n, ctypes.byref(mc),
                                       scratch.data_ptr(), int(repeats), ctypes.byref(b),
                                       ctypes.byref(ms))
        _lib.check(st, self.handle)
        return {"blocks_per_sm": b.value, "ms": ms.value}

    def normals(self, seed: int, n_pairs: int, c1: int = 0, c2: int = 0, c3: int = 9):
        """pdd_normals: (z [2 n_pairs] float32, u [n_pairs] float32) CUDA tensors."""
        z = torch.empty(2 * int(n_pairs), dtype=torch.float32, device=self.device)
        u = torch.empty(int(n_pairs), dtype=torch.float32, device=self.device)
        with torch.cuda.device(self.device):
            self._bind_stream()
            st = self.lib.pdd_normals(self.handle, int(seed) & (2**64 - 1), int(c1), int(c2),
                                      int(c3), int(n_pairs), z.data_ptr(), u.data_ptr())
        _lib.check(st, self.handle)
        return z, u

    def wos_solve(self, nodes, *, seed: int, n_paths: int, eps: float,
                  max_steps: int = 10**6, precision: str = "fp32", path_offset: int = 0,
                  dump_paths: bool = False, diag: bool = False) -> dict:
        """pdd_wos_solve (Walk on Spheres, Laplace problem)."""
        nodes = _dev_f64(nodes, self.device).reshape(-1, 2)
        n = nodes.shape[0]
        mean = torch.empty(n, dtype=_F64, device=self.device)
        se = torch.empty(n, dtype=_F64, device=self.device)
        cnt = torch.empty(n, dtype=_I64, device=self.device)
        wp = _lib.WosParams(int(seed) & (2**64 - 1), int(n_paths), int(path_offset),
                            int(max_steps), float(eps), _lib.PRECISION[precision], 0)
        res = {"mean": mean, "se": se, "n": cnt}
        dg = None
        if diag or dump_paths:
            dg = _lib.Diag()
            if dump_paths:
                res["score"] = torch.empty((n, int(n_paths)), dtype=_F64, device=self.device)
                res["steps"] = torch.empty((n, int(n_paths)), dtype=_I32, device=self.device)
                res["exit"] = torch.empty((n, int(n_paths), 2), dtype=_F64, device=self.device)
                dg.d_path_score = res["score"].data_ptr()
                dg.d_path_steps = res["steps"].data_ptr()
                dg.d_path_exit = res["exit"].data_ptr()
        with torch.cuda.device(self.device):
            self._bind_stream()
            st = self.lib.pdd_wos_solve(self.handle, nodes.data_ptr(), n, ctypes.byref(wp),
                                        mean.data_ptr(), se.data_ptr(), cnt.data_ptr(),
                                        ctypes.byref(dg) if dg is not None else None)
        res["status"] = _lib.check(st, self.handle, allow=(_lib.PDD_OK, _lib.PDD_ECAP))
        if dg is not None:
            res["path_steps"], res["capped"] = int(dg.path_steps), int(dg.capped)
        return res

    def philox_stream(self, seed: int, j0: int, c1: int, c2: int, c3: int, n_blocks: int):
        """pdd_philox_stream: uint32 [n_blocks, 4] CUDA tensor."""
        out = torch.empty((int(n_blocks), 4), dtype=torch.int32, device=self.device)
        with torch.cuda.device(self.device):
            self._bind_stream()
            st = self.lib.pdd_philox_stream(self.handle, int(seed) & (2**64 - 1), int(j0),
                                            int(c1), int(c2), int(c3), int(n_blocks),
                                            out.data_ptr())
        _lib.check(st, self.handle)
        return out


def interface_solve_host(prob: dict, nodes: np.ndarray, **kw) -> dict:
    """End-to-end call with host inputs and outputs: pinned host -> device copy
    of the nodes, pdd_interface_solve, device -> host copy of the results."""
    with Context(prob) as ctx:
        h = torch.from_numpy(np.ascontiguousarray(nodes, dtype=np.float64)).pin_memory()
        r = ctx.interface_solve(h, **kw)
        return {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in r.items()}


class InterfaceValues(torch.autograd.Function):
    """u(nodes; theta, phi) for the Poisson-Fourier family as a differentiable
    function of (theta [64], phi [16]).  Forward: pdd_interface_solve with the
    given parameters.  Backward: pdd_interface_grad with the incoming
    cotangent, on the same random streams (paths re-simulated from their
    Philox keys, nothing stored)."""

    @staticmethod
    def forward(fctx, theta, phi, pdd_ctx, nodes, mc):
        params = torch.cat([theta.detach().reshape(-1), phi.detach().reshape(-1)])
        params = params.to("cpu", torch.float64).numpy()
        pdd_ctx.set_params(params)
        r = pdd_ctx.interface_solve(nodes, precision="fp32", **mc)
        fctx.pdd_ctx, fctx.nodes, fctx.mc, fctx.params = pdd_ctx, nodes, mc, params
        fctx.devices = (theta.device, phi.device)
        fctx.dtypes = (theta.dtype, phi.dtype)
        return r["mean"].clone()

    @staticmethod
    def backward(fctx, grad_u):
        pdd_ctx = fctx.pdd_ctx
        pdd_ctx.set_params(fctx.params)
        g = pdd_ctx.interface_grad(fctx.nodes, grad_out=grad_u.detach().to(torch.float64),
                                   jacobian=False, **fctx.mc)
        dth = g["dtheta"].to(fctx.devices[0], fctx.dtypes[0])
        dph = g["dphi"].to(fctx.devices[1], fctx.dtypes[1])
        return dth, dph, None, None, None


def interface_values(theta, phi, pdd_ctx: Context, nodes, **mc):
    """Differentiable node estimates (see InterfaceValues)."""
    return InterfaceValues.apply(theta, phi, pdd_ctx, nodes, mc)


def laplace_pdd_solve(ctx: Context, *, n_nodes: int = 16, n_paths: int = 10_000, dt: float = 1e-3,
                      seed: int, grid=(129, 129), precision: str = "fp64",
                      method: str = "dst", tol: float = 1e-12) -> dict:
    """The two stages of PDD for the Laplace problem Eq. 1.1 on the unit square
    split at x = 1/2 (Sec. 2.1, Fig. 2.2): stage one estimates u at n_nodes
    interface nodes (1/2, k/(n_nodes+1)) by pdd_interface_solve; stage two
    interpolates them (not-a-knot spline) and solves each half independently
    by pdd_subdomain_solve (by default directly, by sine transforms).  Returns the node estimates and the two subdomain
    grids ([ny][nx] each; they share the interface column x = 1/2)."""
    if ctx.prob["problem"] != "laplace_expcos" or ctx.prob["geometry"] != "unit_square":
        raise ValueError("laplace_pdd_solve needs the Laplace problem on the unit square")
    y = torch.arange(1, n_nodes + 1, dtype=_F64) / (n_nodes + 1)
    nodes = torch.stack([torch.full_like(y, 0.5), y], 1)
    r = ctx.interface_solve(nodes, seed=seed, dt=dt, n_paths=n_paths, precision=precision)
    left = ctx.subdomain_solve((0.0, 0.0), (0.5, 1.0), grid, 0, 1, y, r["mean"], method=method,
                               tol=tol)
    right = ctx.subdomain_solve((0.5, 0.0), (1.0, 1.0), grid, 0, 0, y, r["mean"], method=method,
                                tol=tol)
    return {"nodes": nodes, "mean": r["mean"], "se": r["se"], "left": left["u"],
            "right": right["u"], "iters": left["iters"] + right["iters"],
            "status": max(left["status"], right["status"])}


def elliptic3d_pdd_solve(ctx: Context, nodes, values, node_axis=None, *, grid: int = 129,
                         split: int = 4, n_bnd: int = 32, method: str = "dst",
                         tol: float = 1e-12, max_iter: int = 200) -> dict:
    """Stage two of PDD for the 3-D problem on the unit cube split into
    split^3 subdomains (Sec. 2.1, Fig. 2.2): the node estimates `values` at
    `nodes` (every node on one of the internal planes x_a = k / split) are
    interpolated on each plane (pdd_interface_interp, evaluated on the
    plane's grid of `grid` x `grid` points; node_axis, if given, names the
    plane axis each node belongs to, so that a node on two planes' line of
    intersection is used by its own plane only), and the subdomains are
    solved independently, all in one batched call (pdd_subdomain_solve_batch),
    with the interpolated values on their interface faces and g on the cube's
    boundary.  Returns the global solution
    u [grid, grid, grid] ([z][y][x]), the largest iteration count and
    residual, and the time of each part is left to the caller."""
    if ctx.prob["problem"] != "elliptic_manufactured":
        raise ValueError("elliptic3d_pdd_solve needs the 3-D problem on the unit cube")
    if (grid - 1) % split:
        raise ValueError("grid - 1 must be a multiple of split")
    dev = ctx.device
    nodes = _dev_f64(nodes, dev).reshape(-1, 3)
    values = _dev_f64(values, dev).reshape(-1)
    if node_axis is not None:
        node_axis = torch.as_tensor(node_axis, device=dev).reshape(-1)
    t = torch.linspace(0.0, 1.0, grid, dtype=_F64, device=dev)
    planes, queries = [], []
    for a in range(3):
        for k in range(1, split):
            pos = k / split
            sel = nodes[:, a] == pos
            if node_axis is not None:
                sel &= node_axis == a
            planes.append((a, pos, nodes[sel], values[sel]))
            o = [b for b in range(3) if b != a]
            g2, g1 = torch.meshgrid(t, t, indexing="ij")      # [slow = o[1]][fast = o[0]]
            q = torch.empty((grid * grid, 3), dtype=_F64, device=dev)
            q[:, a] = pos
            q[:, o[0]] = g1.reshape(-1)
            q[:, o[1]] = g2.reshape(-1)
            queries.append(q)
    vals = ctx.interface_interp(planes, queries, n_bnd=n_bnd)
    plane_grid = {(a, k): vals[a * (split - 1) + k - 1].reshape(grid, grid)
                  for a in range(3) for k in range(1, split)}
    m = (grid - 1) // split + 1
    u = torch.empty((grid, grid, grid), dtype=_F64, device=dev)
    boxes, slices = [], []
    for kz in range(split):
        for ky in range(split):
            for kx in range(split):
                kk = (kx, ky, kz)
                lo = [kk[a] / split for a in range(3)]
                hi = [(kk[a] + 1) / split for a in range(3)]
                sl = [slice(kk[a] * (m - 1), kk[a] * (m - 1) + m) for a in range(3)]
                faces = {}
                for a in range(3):
                    o = [b for b in range(3) if b != a]
                    for side in (0, 1):
                        plane = kk[a] + side
                        if 0 < plane < split:
                            pg = plane_grid[(a, plane)]
                            faces[2 * a + side] = pg[sl[o[1]], sl[o[0]]].contiguous()
                boxes.append((lo, hi, faces))
                slices.append(sl)
    # the split^3 subdomains are independent: one batched solve
    r = ctx.subdomain_solve3d_batch(boxes, (m, m, m), method=method, tol=tol, max_iter=max_iter)
    for b, sl in enumerate(slices):
        u[sl[2], sl[1], sl[0]] = r["u"][b]
    return {"u": u, "iters": r["iters"], "resid": r["resid"], "plane_values": plane_grid}
