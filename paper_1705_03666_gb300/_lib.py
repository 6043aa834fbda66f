"""ctypes view of libpdd.so (include/pdd.h).  Argument marshalling only.

Loading fails loudly when the library is missing or a symbol is absent: there
is no CPU or Python fallback for any entry point.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpdd.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "pdd.h")

PDD_OK, PDD_EINVAL, PDD_ENOMEM, PDD_ECUDA, PDD_ETIMEOUT, PDD_ECAP = range(6)
GEOMETRY = {"interval": 0, "unit_square": 1, "l_shape": 2, "unit_cube": 3, "free_space": 4}
PROBLEM = {"laplace_expcos": 1, "elliptic_manufactured": 2, "poisson_fourier": 3, "kpp": 7}
PRECISION = {"fp32": 0, "fp64": 1}
STENCIL = {"cg": 0, "jacobi": 1, "cg_mixed": 2, "dst": 3}


class Problem(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("geometry", ctypes.c_int32),
                ("dim", ctypes.c_int32), ("n_params", ctypes.c_int32),
                ("params", ctypes.POINTER(ctypes.c_double)), ("sigma", ctypes.c_double)]


class MCParams(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("dt", ctypes.c_double),
                ("n_paths", ctypes.c_int64), ("max_steps", ctypes.c_int64),
                ("path_offset", ctypes.c_int64), ("precision", ctypes.c_int32),
                ("bridge", ctypes.c_int32), ("node_offset", ctypes.c_int64)]


class BranchParams(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("n_trees", ctypes.c_int64),
                ("tree_offset", ctypes.c_int64), ("max_particles", ctypes.c_int64),
                ("max_depth", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class GridBranchParams(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("n_trees", ctypes.c_int64),
                ("tree_offset", ctypes.c_int64), ("max_particles", ctypes.c_int64),
                ("max_depth", ctypes.c_int32), ("bridge", ctypes.c_int32),
                ("dt", ctypes.c_double)]


class MlmcParams(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("n_paths", ctypes.c_int64),
                ("max_steps", ctypes.c_int64), ("dt0", ctypes.c_double),
                ("level", ctypes.c_int32), ("refine", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("bridge", ctypes.c_int32)]


class Subdomain(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("n", ctypes.c_int32 * 3), ("iface_axis", ctypes.c_int32),
                ("iface_side", ctypes.c_int32), ("method", ctypes.c_int32),
                ("max_iter", ctypes.c_int64), ("tol", ctypes.c_double)]


class BatchNodes(ctypes.Structure):
    _fields_ = [("d_nodes", ctypes.c_void_p), ("d_problem", ctypes.c_void_p),
                ("d_dt", ctypes.c_void_p), ("n", ctypes.c_int64)]


class BatchParams(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("n_pilot", ctypes.c_int64),
                ("n_min", ctypes.c_int64), ("n_max", ctypes.c_int64),
                ("target_se", ctypes.c_double), ("max_steps", ctypes.c_int64),
                ("chunk", ctypes.c_int32), ("bridge", ctypes.c_int32)]


class WosParams(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("n_paths", ctypes.c_int64),
                ("path_offset", ctypes.c_int64), ("max_steps", ctypes.c_int64),
                ("eps", ctypes.c_double), ("precision", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class Diag(ctypes.Structure):
    _fields_ = [("d_path_score", ctypes.c_void_p), ("d_path_steps", ctypes.c_void_p),
                ("d_path_aux", ctypes.c_void_p), ("path_steps", ctypes.c_int64),
                ("capped", ctypes.c_int64), ("d_path_exit", ctypes.c_void_p),
                ("d_node_flags", ctypes.c_void_p)]


# per-node flags (pdd_diag.d_node_flags)
NODE_FLAGS = {"on_boundary": 1, "outside": 2, "capped": 4, "discarded": 8, "empty": 16,
              "se_unmet": 32}


_lock = threading.Lock()
_lib = None

_VP, _I64, _U32, _U64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
_SIGS = {
    "pdd_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Problem),
                                  ctypes.c_int, _VP]),
    "pdd_set_stream": (ctypes.c_int, [_VP, _VP]),
    "pdd_set_tuning": (ctypes.c_int, [_VP, ctypes.c_int, _I64]),
    "pdd_interface_solve": (ctypes.c_int, [_VP, _VP, _I64, ctypes.POINTER(MCParams), _VP, _VP,
                                           _VP, ctypes.POINTER(Diag)]),
    "pdd_profile": (ctypes.c_int, [_VP, ctypes.c_int]),
    "pdd_profile_read": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int64)]),
    "pdd_branching_solve": (ctypes.c_int, [_VP, _VP, _I64, ctypes.POINTER(BranchParams), _VP,
                                           _VP, _VP, ctypes.POINTER(Diag)]),
    "pdd_subdomain_solve": (ctypes.c_int, [_VP, ctypes.POINTER(Subdomain), _VP, _VP, _I64, _VP,
                                           ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(ctypes.c_double)]),
    "pdd_subdomain_solve_batch": (ctypes.c_int, [_VP, ctypes.POINTER(Subdomain), ctypes.c_int32,
                                                 _VP, _I64, _VP, ctypes.POINTER(ctypes.c_int64),
                                                 ctypes.POINTER(ctypes.c_double),
                                                 ctypes.POINTER(ctypes.c_int64),
                                                 ctypes.POINTER(ctypes.c_double)]),
    "pdd_interface_grad": (ctypes.c_int, [_VP, _VP, _I64, ctypes.POINTER(MCParams), _VP, _VP,
                                          _VP, _VP, _VP, ctypes.POINTER(Diag)]),
    "pdd_set_params": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.c_int32]),
    "pdd_interface_solve_static": (ctypes.c_int, [ctypes.POINTER(Problem), ctypes.c_int, _VP,
                                                   _VP, _I64, ctypes.POINTER(MCParams), _VP,
                                                   _VP, _VP]),
    "pdd_batch_solve": (ctypes.c_int, [_VP, ctypes.POINTER(Problem), ctypes.c_int32,
                                       ctypes.POINTER(BatchNodes), ctypes.POINTER(BatchParams),
                                       _VP, _VP, _VP, ctypes.c_int32, ctypes.POINTER(Diag)]),
    "pdd_interface_solve_naive": (ctypes.c_int, [_VP, _VP, _I64, ctypes.POINTER(MCParams), _VP,
                                                 _VP, _VP]),
    "pdd_autotune": (ctypes.c_int, [_VP, _VP, _I64, ctypes.POINTER(MCParams), _VP, ctypes.c_int32,
                                    ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_double)]),
    "pdd_autotune_batch": (ctypes.c_int, [_VP, ctypes.POINTER(Problem), ctypes.c_int32,
                                          ctypes.POINTER(BatchNodes), ctypes.POINTER(BatchParams),
                                          _VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_double)]),
    "pdd_normals": (ctypes.c_int, [_VP, _U64, _U32, _U32, _U32, _I64, _VP, _VP]),
    "pdd_wos_solve": (ctypes.c_int, [_VP, _VP, _I64, ctypes.POINTER(WosParams), _VP, _VP, _VP,
                                     ctypes.POINTER(Diag)]),
    "pdd_branching_grid_solve": (ctypes.c_int, [_VP, _VP, _I64, _VP, ctypes.c_int32,
                                                ctypes.POINTER(GridBranchParams), _VP, _VP, _VP,
                                                ctypes.POINTER(Diag)]),
    "pdd_mlmc_level": (ctypes.c_int, [_VP, _VP, _I64, ctypes.POINTER(MlmcParams), _VP, _VP, _VP,
                                      _VP, ctypes.POINTER(Diag)]),
    "pdd_mlmc_solve": (ctypes.c_int, [_VP, _VP, _I64, ctypes.POINTER(MlmcParams), ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_int64), _VP, _VP, _VP, _VP,
                                      ctypes.POINTER(Diag)]),
    "pdd_interface_interp": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_int64), _VP, _VP,
                                            ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), _VP,
                                            _VP]),
    "pdd_philox_stream": (ctypes.c_int, [_VP, _U64, _U32, _U32, _U32, _U32, _I64, _VP]),
    "pdd_destroy": (None, [_VP]),
    "pdd_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "pdd_last_error": (ctypes.c_char_p, [_VP]),
}


def header_symbols() -> list[str]:
    """Names of the functions include/pdd.h declares."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"PDD_API\s+[\w\s\*]*?\b(pdd_\w+)\s*\(", text)))


def load() -> ctypes.CDLL:
    """Load libpdd.so (it must have been built, e.g. by __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"libpdd.so not found at {LIB_PATH}: build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'` (no fallback exists)")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)  # AttributeError if the symbol is missing
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class PDDError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"pdd status {status}: {message}")
        self.status = status


def check(status: int, ctx=None, allow=(PDD_OK,), create: bool = False) -> int:
    """Raise PDDError unless status is allowed; the message adds the
    context's last error, or (create=True) why pdd_create failed."""
    if status in allow:
        return status
    lib = load()
    msg = lib.pdd_status_string(status).decode()
    if ctx or create:
        extra = lib.pdd_last_error(ctx if ctx else None).decode()
        if extra:
            msg = f"{msg}: {extra}"
    raise PDDError(status, msg)
