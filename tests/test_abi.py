"""C-ABI checks that need no GPU: the library builds, loads, and exports every
function include/pdd.h declares; the Python binding covers the same set."""
import ctypes
import subprocess

import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_1705_03666_gb300 import build as b
    b.build()
    from paper_1705_03666_gb300 import _lib
    return _lib


def test_header_symbols_exported(lib):
    names = lib.header_symbols()
    assert "pdd_interface_solve" in names and "pdd_create" in names
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in names if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    # nothing but the C ABI is exported
    assert all(n.startswith("pdd_") for n in exported), sorted(exported)


def test_binding_matches_header(lib):
    assert sorted(lib._SIGS) == lib.header_symbols()
    cdll = lib.load()
    for n in lib.header_symbols():
        assert getattr(cdll, n) is not None


def test_status_strings_without_gpu(lib):
    cdll = lib.load()
    assert cdll.pdd_status_string(0) == b"ok"
    assert cdll.pdd_status_string(5).startswith(b"some paths")


def test_create_rejects_invalid_problem_without_gpu(lib):
    """Argument checks run before any device call."""
    import numpy as np
    cdll = lib.load()
    params = np.zeros(1)
    bad = lib.Problem(2, 1, 3, 0, params.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1.0)
    h = ctypes.c_void_p()
    assert cdll.pdd_create(ctypes.byref(h), ctypes.byref(bad), 0, None) == lib.PDD_EINVAL
    neg = lib.Problem(1, 1, 2, 0, params.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), -1.0)
    assert cdll.pdd_create(ctypes.byref(h), ctypes.byref(neg), 0, None) == lib.PDD_EINVAL
    # KPP with q not summing to one (Assumption 3.1)
    kp = np.array([1.0, 1.0, 4.0, 2.0, 0.0, 0.0, 0.5, 0.0, 0.0, 0.5])
    kpp = lib.Problem(7, 4, 2, kp.size, kp.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1.0)
    assert cdll.pdd_create(ctypes.byref(h), ctypes.byref(kpp), 0, None) == lib.PDD_EINVAL
    # the reason is kept per thread and read with a NULL context
    assert cdll.pdd_last_error(None) == b"q must sum to 1"
    assert cdll.pdd_create(ctypes.byref(h), ctypes.byref(neg), 0, None) == lib.PDD_EINVAL
    assert cdll.pdd_last_error(None) == b"sigma must be > 0"
    assert cdll.pdd_create(ctypes.byref(h), ctypes.byref(bad), 0, None) == lib.PDD_EINVAL
    assert cdll.pdd_last_error(None) == b"ELLIPTIC_MANUFACTURED needs dim 3 on the unit cube"
    assert cdll.pdd_create(None, ctypes.byref(neg), 0, None) == lib.PDD_EINVAL
    assert cdll.pdd_last_error(None) == b"out or problem is NULL"
    ok = lib.Problem(1, 1, 2, 0, params.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1.0)
    assert cdll.pdd_create(ctypes.byref(h), ctypes.byref(ok), -1, None) == lib.PDD_EINVAL
    assert cdll.pdd_last_error(None) == b"device must be >= 0"
    with pytest.raises(lib.PDDError, match="sigma must be > 0"):
        lib.check(lib.PDD_EINVAL if cdll.pdd_create(ctypes.byref(h), ctypes.byref(neg), 0, None)
                  else lib.PDD_OK, create=True)


def test_struct_layouts(lib):
    assert ctypes.sizeof(lib.Problem) == 32
    assert ctypes.sizeof(lib.MCParams) == 56
    assert ctypes.sizeof(lib.Diag) == 56
    assert ctypes.sizeof(lib.BranchParams) == 40
    assert ctypes.sizeof(lib.Subdomain) == 88
    assert ctypes.sizeof(lib.WosParams) == 48
    assert ctypes.sizeof(lib.GridBranchParams) == 48
    assert ctypes.sizeof(lib.MlmcParams) == 48


def test_struct_layouts_match_c_compiler(lib, tmp_path):
    """Every ctypes structure of the binding has the size and field offsets
    that a C compiler gives the header's struct."""
    import os
    structs = {"Problem": "pdd_problem", "MCParams": "pdd_mc_params", "Diag": "pdd_diag",
               "BranchParams": "pdd_branch_params", "GridBranchParams": "pdd_grid_branch_params",
               "MlmcParams": "pdd_mlmc_params", "Subdomain": "pdd_subdomain",
               "BatchNodes": "pdd_batch_nodes", "BatchParams": "pdd_batch_params",
               "WosParams": "pdd_wos_params"}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pdd.h"', "int main(void) {"]
    expect = []
    for py, c in structs.items():
        cls = getattr(lib, py)
        lines.append(f'  printf("%zu\\n", sizeof({c}));')
        expect.append(ctypes.sizeof(cls))
        for name, _ in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({c}, {name}));')
            expect.append(getattr(cls, name).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert got == expect


def test_enum_values_match_header(lib):
    """The binding's tables of geometry, problem, precision, stencil method
    and status codes carry the values include/pdd.h gives them."""
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "include", "pdd.h")).read()
    vals = {m.group(1): int(m.group(2))
            for m in re.finditer(r"\b(PDD_[A-Z0-9_]+)\s*=\s*(\d+)", hdr)}
    tables = [(lib.GEOMETRY, "PDD_GEOM_"), (lib.PROBLEM, "PDD_PROB_"),
              (lib.PRECISION, "PDD_"), (lib.STENCIL, "PDD_STENCIL_")]
    for table, prefix in tables:
        for name, v in table.items():
            assert vals[prefix + name.upper()] == v, (prefix + name.upper(), v)
    for name in ("PDD_OK", "PDD_EINVAL", "PDD_ENOMEM", "PDD_ECUDA", "PDD_ETIMEOUT", "PDD_ECAP"):
        assert vals[name] == getattr(lib, name), name
    for name, v in lib.NODE_FLAGS.items():
        assert vals["PDD_NODE_" + name.upper()] == v, name
