"""The C ABI library loads and exports every symbol that include/dms.h
declares (no compute calls: these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dms.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dms_[a-z_]+)\s*\(", src)))


def test_header_declares_the_entry_points():
    names = _declared()
    for want in ("dms_grid_create", "dms_compute_diagram", "dms_get_counts",
                 "dms_fetch_pairs", "dms_grid_destroy", "dms_status_string"):
        assert want in names


def test_library_exports_every_declared_symbol():
    import paper_2206_13932_gb300 as dms
    path = dms.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    import paper_2206_13932_gb300 as dms
    lib = dms.load(build_if_missing=True)
    for code in range(8):
        assert lib.dms_status_string(code)
    assert lib.dms_status_string(99) == b"unknown status"


def test_pair_record_layout():
    import paper_2206_13932_gb300 as dms
    assert dms.PAIR_DTYPE.itemsize == 56
    assert [dms.PAIR_DTYPE.fields[f][1] for f in ("birth_simplex", "death_simplex",
                                                  "birth_vertex", "death_vertex",
                                                  "birth_bits", "death_bits", "dim",
                                                  "essential")] == [0, 8, 16, 24, 32, 40, 48, 49]


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    """The binding raises instead of computing anything when libdms is absent."""
    import paper_2206_13932_gb300 as dms
    monkeypatch.setattr(dms, "_LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(dms, "_lib", None)
    with pytest.raises(RuntimeError):
        dms.load()
