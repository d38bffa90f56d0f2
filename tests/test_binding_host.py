"""Argument marshalling of the Python binding, on the host (no GPU): the
pointer, host flag and size checks that ``Grid`` and ``Batch`` hand to the C
ABI.  The handles are built without ``dms_grid_create`` (no device); only
their marshalling methods run."""
import numpy as np
import pytest

import paper_2206_13932_gb300 as dms


def _grid(shape_xyz, dtype):
    g = object.__new__(dms.Grid)
    g.shape_xyz, g.dtype = tuple(shape_xyz), np.dtype(dtype)
    return g


def _batch(shapes, dtype):
    b = object.__new__(dms.Batch)
    b.shapes_xyz = [tuple(s) for s in shapes]
    b.dtype = np.dtype(dtype)
    b.sizes = [x * y * z for x, y, z in b.shapes_xyz]
    b.n = sum(b.sizes)
    return b


def test_grid_takes_a_host_array_of_its_shape_and_dtype():
    g = _grid((4, 3, 2), np.float32)
    v = np.arange(24, dtype=np.float32).reshape(2, 3, 4)
    ptr, on_host, keep = g._field_ptr(v)
    assert on_host == 1 and ptr == keep.ctypes.data and np.array_equal(keep, v)
    with pytest.raises(ValueError):
        g._field_ptr(np.zeros((2, 3, 5), np.float32))        # wrong size
    with pytest.raises(ValueError):
        g._field_ptr(np.zeros((2, 3, 4), np.float64))        # wrong dtype


def test_grid_takes_a_cpu_tensor_as_host_memory():
    torch = pytest.importorskip("torch")
    g = _grid((4, 3, 2), np.float32)
    t = torch.arange(24, dtype=torch.float32).reshape(2, 3, 4)
    ptr, on_host, keep = g._field_ptr(t)
    assert on_host == 1 and ptr == t.data_ptr()
    with pytest.raises(TypeError):
        g._field_ptr(t.double())
    with pytest.raises(ValueError):
        g._field_ptr(t.transpose(0, 2))                      # not contiguous


def test_batch_packs_its_fields_in_order():
    shapes = [(2, 2, 2), (3, 1, 2), (1, 1, 1)]
    b = _batch(shapes, np.uint16)
    fields = [np.full((z, y, x), k, np.uint16) for k, (x, y, z) in enumerate(shapes)]
    ptr, on_host, keep = b._field_ptr(fields)
    assert on_host == 1 and keep.size == b.n
    assert list(keep) == [0] * 8 + [1] * 6 + [2]
    with pytest.raises(ValueError):
        b._field_ptr(fields[:2])                             # a field missing
    with pytest.raises(ValueError):
        b._field_ptr([f.astype(np.float32) for f in fields])  # wrong dtype


def test_batch_reshape_wants_a_list_of_shapes():
    b = _batch([(2, 2, 2)], np.float32)
    with pytest.raises(dms.DmsError):
        b.reshape((2, 2, 2))
