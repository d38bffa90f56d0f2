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


def test_argument_checks_without_gpu():
    """Invalid arguments are refused before any CUDA call, so these run on a
    machine without a GPU: every entry point rejects a null handle, and
    dms_grid_create rejects bad sizes, dtypes and options."""
    import paper_2206_13932_gb300 as dms
    lib = dms.load(build_if_missing=True)
    bad = 1   # DMS_ERR_INVALID_ARG
    h = ctypes.c_void_p()

    def create(nx, ny, nz, dtype=1, opts=None):
        return lib.dms_grid_create(nx, ny, nz, dtype, ctypes.byref(opts) if opts else None,
                                   ctypes.byref(h))

    assert create(0, 4, 4) == bad and create(4, -1, 4) == bad
    assert create(1 << 16, 1 << 16, 1) == bad            # nx*ny >= 2^31
    assert create(1 << 11, 1 << 10, 1 << 10) == bad      # N >= 2^31
    assert create(4, 4, 4, dtype=3) == bad
    assert create(4, 4, 4, opts=dms._Options(2, 0, 0)) == bad    # virtual maximum neither 0 nor 1
    assert create(4, 4, 4, opts=dms._Options(1, -1, 0)) == bad    # negative iteration cap
    assert create(4, 4, 4, opts=dms._Options(1, 0, 4)) == bad    # unknown D1 mode
    assert create(4, 4, 4, opts=dms._Options(1, 0, 0, 2)) == bad  # generators neither 0 nor 1
    assert create(4, 4, 4, opts=dms._Options(1, 0, 3, 1)) == bad  # generators need the traced mode
    assert create(1 << 10, 1 << 10, 300, opts=dms._Options(1, 0, 0, 1)) == bad  # 7N >= 2^31
    shapes = (ctypes.c_int64 * 3)(4, 4, 4)
    assert lib.dms_batch_create(1, shapes, 1, ctypes.byref(dms._Options(1, 0, 0, 1)),
                                ctypes.byref(h)) == bad          # generators: single grids
    assert lib.dms_grid_create(4, 4, 4, 1, None, None) == bad     # no output handle
    assert not h.value
    null = ctypes.c_void_p(0)
    p3, p4 = (ctypes.c_int64 * 3)(), (ctypes.c_int64 * 4)()
    w = ctypes.c_int64(0)
    assert lib.dms_compute_diagram(null, null, 1, null) == bad
    assert lib.dms_get_counts(null, p3, p4) == bad
    assert lib.dms_fetch_pairs(null, 0, null, 0, ctypes.byref(w), 0) == bad
    assert lib.dms_grid_reshape(null, 4, 4, 4) == bad
    assert lib.dms_batch_reshape(null, 1, p3) == bad
    assert lib.dms_batch_offsets(null, 0, p4) == bad
    assert lib.dms_backward_pairs(null, 0, 0, null, null, null, null) == bad
    r = ctypes.c_uint64(0)
    assert lib.dms_get_result_id(null, ctypes.byref(r)) == bad
    assert lib.dms_fetch_generators(null, null, 0, ctypes.byref(w)) == bad
    assert lib.dms_get_stage_ms(null, (ctypes.c_float * 8)()) == bad
    assert lib.dms_get_kernel_ms(null, (ctypes.c_float * 12)()) == bad
    assert lib.dms_get_stats(null, (ctypes.c_int64 * 16)()) == bad
    assert lib.dms_get_work(null, (ctypes.c_int64 * 4)()) == bad
    assert lib.dms_get_device_bytes(null, ctypes.byref(w)) == bad
    assert lib.dms_set_tuning(null, (ctypes.c_int32 * 10)(), 10) == bad
    assert lib.dms_get_tuning(null, (ctypes.c_int32 * 10)(), 10) == bad
    assert lib.dms_grid_destroy(null) == bad
    assert lib.dms_batch_create(1, None, 1, None, ctypes.byref(h)) == bad
    # the allocation-free classification checks its arguments first too
    n = ctypes.c_int64(0)
    buf = (ctypes.c_uint8 * 64)()
    crit = (ctypes.c_int32 * 64)()
    cls = lib.dms_classify_static
    assert cls(None, 1, 4, 4, 4, buf, crit, 64, ctypes.byref(n), None) == bad
    assert cls(buf, 1, 4, 4, 4, None, crit, 64, ctypes.byref(n), None) == bad
    assert cls(buf, 1, 4, 4, 4, buf, None, 64, ctypes.byref(n), None) == bad
    assert cls(buf, 1, 4, 4, 4, buf, crit, -1, ctypes.byref(n), None) == bad
    assert cls(buf, 1, 0, 4, 4, buf, crit, 64, ctypes.byref(n), None) == bad
    assert cls(buf, 1, 1 << 10, 1 << 10, 1 << 9, buf, crit, 64, ctypes.byref(n), None) == bad
    assert cls(buf, 7, 4, 4, 4, buf, crit, 64, ctypes.byref(n), None) == bad


def test_batch_shapes_are_checked_without_gpu():
    """dms_batch_create refuses bad field lists before any CUDA call."""
    import paper_2206_13932_gb300 as dms
    lib = dms.load(build_if_missing=True)
    h = ctypes.c_void_p()

    def create(shapes):
        flat = (ctypes.c_int64 * max(1, len(shapes) * 3))(*[v for s in shapes for v in s])
        return lib.dms_batch_create(len(shapes), flat, 1, None, ctypes.byref(h))

    assert create([]) == 1                                   # no field
    assert create([(4, 4, 4), (0, 4, 4)]) == 1               # an empty axis
    assert create([(1 << 16, 1 << 16, 1)]) == 1              # nx*ny >= 2^31
    assert create([(1 << 10, 1 << 10, 1 << 10)] * 2) == 1    # total >= 2^31
    assert create([(2, 2, 2)] * 65536) == 1                  # more fields than the index holds
    assert not h.value
