"""The product path and the oracle share no code and the product never falls
back to the oracle: no module of the package imports or loads it, neither
side includes the other's sources, and a missing libpdd.so is an error."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1705_03666_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _sources(top, exts):
    for d, dirs, files in os.walk(top):
        dirs[:] = [x for x in dirs if x not in ("__pycache__", "_build")]
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_package_never_loads_the_oracle():
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b)|liborc|orc_\w+\s*\(|oracle/", re.M)
    hits = []
    for p in _sources(PKG, (".py", ".cu", ".cuh", ".hpp", ".h")):
        text = open(p, encoding="utf-8").read()
        for m in pat.finditer(text):
            hits.append(f"{os.path.relpath(p, ROOT)}: {m.group(0).strip()}")
    assert not hits, hits


def test_no_shared_sources():
    # the oracle includes only the C library; the kernels include only their
    # own headers and CUDA's
    orc_inc = set()
    for p in _sources(ORACLE, (".c", ".h")):
        orc_inc |= set(re.findall(r'#include\s*[<"]([^>"]+)[>"]', open(p).read()))
    assert orc_inc, "oracle sources not found"
    assert all("/" not in h and not h.endswith((".cuh", ".hpp")) for h in orc_inc), orc_inc
    assert "pdd.h" not in orc_inc
    for p in _sources(os.path.join(PKG, "csrc"), (".cu", ".cuh", ".hpp")):
        for h in re.findall(r'#include\s*"([^"]+)"', open(p).read()):
            assert "oracle" not in h and not h.endswith(".c"), (p, h)
    # the Python side of the oracle imports nothing from the package
    orc_py = open(os.path.join(ORACLE, "__init__.py")).read()
    assert not re.search(r"^\s*(from|import)\s+(paper_1705_03666_gb300|\.\.)", orc_py, re.M)
    assert "libpdd" not in orc_py


def test_missing_library_is_an_error(monkeypatch, tmp_path):
    from paper_1705_03666_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libpdd.so"))
    with pytest.raises(RuntimeError, match="no fallback"):
        _lib.load()
