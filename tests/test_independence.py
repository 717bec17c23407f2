"""The oracle and the CUDA path share nothing, and the product path has no fallback (CPU only).

The package (Python binding, C ABI, kernels) neither imports, includes, links nor loads
anything under oracle/; the oracle includes only C library headers; and the binding raises
instead of computing anything when its library is missing.
"""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2106_07575_gb300")


def _package_sources():
    pats = ("*.py", "csrc/*.cu", "csrc/*.cuh", "csrc/*.h", "csrc/*.cpp")
    files = [f for p in pats for f in glob.glob(os.path.join(PKG, p))]
    files += glob.glob(os.path.join(ROOT, "include", "*.h"))
    assert len(files) > 20
    return files


def test_package_never_reaches_the_oracle():
    """No import of the oracle package, no include of its source, no load of its library."""
    bad = re.compile(r"^\s*(import\s+oracle|from\s+oracle)|#\s*include\s*[<\"][^>\"]*(orc|oracle)|liborc|orc\.c\b",
                     re.M)
    hits = [f for f in _package_sources() if bad.search(open(f, encoding="utf-8").read())]
    assert not hits, hits


def test_oracle_includes_only_the_c_library():
    src = open(os.path.join(ROOT, "oracle", "orc.c")).read()
    headers = set(re.findall(r"#\s*include\s*[<\"]([^>\"]+)[>\"]", src))
    assert headers <= {"complex.h", "math.h", "stdlib.h", "string.h", "omp.h"}, headers
    imports = re.compile(r"^\s*(import|from)\s+(paper_2106_07575_gb300|torch)\b|libpty", re.M)
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        assert not imports.search(open(f).read()), f


def test_binding_raises_without_its_library(monkeypatch, tmp_path):
    from paper_2106_07575_gb300 import build, pty

    monkeypatch.setattr(pty, "_lib", None)
    monkeypatch.setattr(build, "lib_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="libpty not built"):
        pty.load(build_if_missing=False)
