"""The product and the oracle stay apart, and the product has no CPU path.

- No module of the package imports the oracle, and the oracle imports nothing
  of the package; no C/CUDA source of one includes a file of the other.
- Without a GPU the package refuses to compute (a status error), instead of
  computing anything on the host.
"""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2206_13932_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _files(top, exts):
    for base, dirs, files in os.walk(top):
        dirs[:] = [d for d in dirs if not d.startswith(("_build", "__pycache__"))]
        for f in files:
            if f.endswith(exts):
                yield os.path.join(base, f)


def test_package_never_imports_the_oracle():
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b)", re.M)
    for f in _files(PKG, (".py",)):
        assert not pat.search(open(f).read()), f


def test_oracle_never_imports_the_package():
    pat = re.compile(r"^\s*(import|from)\s+paper_2206_13932_gb300|^\s*(import|from)\s+\.\.|"
                     r"libdms|ctypes\.CDLL\((?!build\(\))", re.M)
    for f in _files(ORACLE, (".py",)):
        assert not pat.search(open(f).read()), f


def test_no_source_includes_the_other_side():
    inc = re.compile(r'^\s*#\s*include\s*"([^"]+)"', re.M)
    for f in _files(ORACLE, (".c", ".h")):
        for name in inc.findall(open(f).read()):
            assert os.path.dirname(os.path.abspath(os.path.join(os.path.dirname(f), name))) == \
                ORACLE, (f, name)
    for f in list(_files(PKG, (".cu", ".cuh", ".h"))) + [os.path.join(ROOT, "include", "dms.h")]:
        for name in inc.findall(open(f).read()):
            assert "oracle" not in name, (f, name)


def test_compute_without_a_gpu_is_an_error():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2206_13932_gb300 as dms
    dms.load(build_if_missing=True)
    with pytest.raises(dms.DmsError):
        dms.Grid((8, 8, 8), np.float32)
