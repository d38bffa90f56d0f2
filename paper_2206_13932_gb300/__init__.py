"""GB300-native Discrete Morse Sandwich: persistence diagrams D0, D1, D2 of a
PL scalar field on a 3D grid (Freudenthal triangulation), computed on one GPU.

This module is a thin binding of the C ABI in ``include/dms.h`` (library
``_build/libdms.so``): argument marshalling only, every step of the method runs
in the CUDA kernels of ``csrc/``.  PyTorch is used for device memory and
streams.  There is no CPU fallback: if the library is missing the calls raise.

- :class:`Grid` -- one grid shape and dtype; ``compute``, ``fetch``,
  ``reshape``, timings, statistics and ``device_bytes``.
- :class:`Batch` -- many fields of their own shapes in one pass.
- :func:`diagram` -- one field's D0, D1, D2 in one call.
- :func:`classify_static` -- the allocation-free classification step.
- Submodules: ``autograd`` (differentiable births and deaths), ``serve``
  (continuous-batching server), ``autotune`` (launch shapes), ``replicas``
  (timing of independent replicas).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from ._build_lib import LIB as _LIB_PATH
from ._build_lib import build

__all__ = ["build", "load", "Grid", "Batch", "diagram", "classify_static", "PAIR_DTYPE", "DmsError",
           "STATUS"]

PAIR_DTYPE = np.dtype([("birth_simplex", "<i8"), ("death_simplex", "<i8"),
                       ("birth_vertex", "<i8"), ("death_vertex", "<i8"),
                       ("birth_bits", "<u8"), ("death_bits", "<u8"),
                       ("dim", "u1"), ("essential", "u1"), ("pad", "V6")])
assert PAIR_DTYPE.itemsize == 56

STATUS = {0: "DMS_OK", 1: "DMS_ERR_INVALID_ARG", 2: "DMS_ERR_NAN", 3: "DMS_ERR_OOM",
          4: "DMS_ERR_CUDA", 5: "DMS_ERR_ITER_LIMIT", 6: "DMS_ERR_STATE",
          7: "DMS_ERR_CAPACITY"}
_DTYPE_CODE = {np.dtype(np.uint16): 0, np.dtype(np.float32): 1, np.dtype(np.float64): 2}


class DmsError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}")


class _Options(ctypes.Structure):
    _fields_ = [("virtual_max", ctypes.c_int), ("max_iters", ctypes.c_int64),
                ("d1_mode", ctypes.c_int), ("generators", ctypes.c_int)]


_lock = threading.Lock()
_lib = None


def load(build_if_missing: bool = False):
    """The loaded libdms (ctypes).  Raises if it is not built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                if not build_if_missing:
                    raise RuntimeError(f"libdms is not built ({_LIB_PATH}); run build()")
                build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64, vp, p64 = ctypes.c_int64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
            lib.dms_grid_create.argtypes = [i64, i64, i64, ctypes.c_int,
                                            ctypes.POINTER(_Options), ctypes.POINTER(vp)]
            lib.dms_compute_diagram.argtypes = [vp, vp, ctypes.c_int, vp]
            lib.dms_get_counts.argtypes = [vp, p64, p64]
            lib.dms_fetch_pairs.argtypes = [vp, ctypes.c_int, vp, i64, p64, ctypes.c_int]
            lib.dms_get_stage_ms.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
            lib.dms_get_stats.argtypes = [vp, p64]
            lib.dms_get_work.argtypes = [vp, p64]
            lib.dms_get_work.restype = ctypes.c_int
            lib.dms_get_kernel_ms.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
            lib.dms_get_device_bytes.argtypes = [vp, p64]
            lib.dms_get_device_bytes.restype = ctypes.c_int
            lib.dms_classify_static.argtypes = [vp, ctypes.c_int, i64, i64, i64, vp, vp, i64,
                                                p64, vp]
            lib.dms_classify_static.restype = ctypes.c_int
            lib.dms_backward_pairs.argtypes = [vp, ctypes.c_int, ctypes.c_uint64, vp, vp, vp, vp]
            lib.dms_backward_pairs.restype = ctypes.c_int
            lib.dms_get_result_id.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
            lib.dms_get_result_id.restype = ctypes.c_int
            lib.dms_fetch_generators.argtypes = [vp, vp, i64, p64]
            lib.dms_fetch_generators.restype = ctypes.c_int
            lib.dms_grid_reshape.argtypes = [vp, i64, i64, i64]
            lib.dms_grid_reshape.restype = ctypes.c_int
            lib.dms_batch_create.argtypes = [i64, p64, ctypes.c_int, ctypes.POINTER(_Options),
                                             ctypes.POINTER(vp)]
            lib.dms_batch_create.restype = ctypes.c_int
            lib.dms_batch_reshape.argtypes = [vp, i64, p64]
            lib.dms_batch_reshape.restype = ctypes.c_int
            lib.dms_batch_offsets.argtypes = [vp, ctypes.c_int, p64]
            lib.dms_batch_offsets.restype = ctypes.c_int
            p32 = ctypes.POINTER(ctypes.c_int32)
            lib.dms_set_tuning.argtypes = [vp, p32, ctypes.c_int]
            lib.dms_set_tuning.restype = ctypes.c_int
            lib.dms_get_tuning.argtypes = [vp, p32, ctypes.c_int]
            lib.dms_get_tuning.restype = ctypes.c_int
            lib.dms_grid_destroy.argtypes = [vp]
            lib.dms_status_string.argtypes = [ctypes.c_int]
            lib.dms_status_string.restype = ctypes.c_char_p
            for f in ("dms_grid_create", "dms_compute_diagram", "dms_get_counts",
                      "dms_fetch_pairs", "dms_get_stage_ms", "dms_get_stats", "dms_get_kernel_ms",
                      "dms_grid_destroy"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def _check(st: int, where: str):
    if st != 0:
        raise DmsError(st, where)


class Grid:
    """A handle of ``dms_grid``: one grid shape and dtype, reusable across fields.
    ``virtual_max=False`` drops the virtual maximum on the outer boundary
    (App. A): unpaired maxima are then infinite classes of dimension 3,
    listed at the end of ``fetch(2)``.  ``generators=True`` also computes a
    persistent 1-cycle generator of every D1 pair (``generators()``)."""

    def __init__(self, shape_xyz, dtype, max_iters: int = 0, d1_mode: int = 0,
                 virtual_max: bool = True, generators: bool = False):
        self._lib = load()
        self.shape_xyz = tuple(int(s) for s in shape_xyz)
        self.dtype = np.dtype(dtype)
        if self.dtype not in _DTYPE_CODE:
            raise TypeError(f"unsupported dtype {self.dtype}")
        opts = _Options(int(bool(virtual_max)), int(max_iters), int(d1_mode),
                        int(bool(generators)))
        h = ctypes.c_void_p()
        nx, ny, nz = self.shape_xyz
        _check(self._lib.dms_grid_create(nx, ny, nz, _DTYPE_CODE[self.dtype],
                                         ctypes.byref(opts), ctypes.byref(h)),
               "dms_grid_create")
        self._h = h

    def reshape(self, shape_xyz):
        """Reuses this handle (and its device buffers) for another grid shape."""
        shape_xyz = tuple(int(s) for s in shape_xyz)
        _check(self._lib.dms_grid_reshape(self._h, *shape_xyz), "dms_grid_reshape")
        self.shape_xyz = shape_xyz
        return self

    def close(self):
        if getattr(self, "_h", None):
            self._lib.dms_grid_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _field_ptr(self, values):
        """(pointer, on_host, keepalive) for a torch tensor or numpy array."""
        nx, ny, nz = self.shape_xyz
        try:
            import torch
        except ImportError:  # pragma: no cover
            torch = None
        if torch is not None and isinstance(values, torch.Tensor):
            if values.numel() != nx * ny * nz or not values.is_contiguous():
                raise ValueError("field must be contiguous with nx*ny*nz elements")
            if np.dtype(str(values.dtype).replace("torch.", "")) != self.dtype:
                raise TypeError("dtype mismatch")
            return values.data_ptr(), (0 if values.is_cuda else 1), values
        arr = np.ascontiguousarray(values)
        if arr.size != nx * ny * nz or arr.dtype != self.dtype:
            raise ValueError("field size or dtype mismatch")
        return arr.ctypes.data, 1, arr

    def compute(self, values, stream=None):
        """Runs the pipeline on ``values`` (torch CUDA tensor: device pointer;
        numpy array or CPU tensor: host pointer copied in on the stream)."""
        ptr, on_host, keep = self._field_ptr(values)
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
            except ImportError:  # pragma: no cover
                stream = 0
        _check(self._lib.dms_compute_diagram(self._h, ctypes.c_void_p(ptr), on_host,
                                             ctypes.c_void_p(int(stream))),
               "dms_compute_diagram")
        del keep
        return self

    def counts(self):
        p = (ctypes.c_int64 * 3)()
        e = (ctypes.c_int64 * 4)()
        _check(self._lib.dms_get_counts(self._h, p, e), "dms_get_counts")
        return tuple(p), tuple(e)

    def list_rows(self, dim: int) -> int:
        """Rows that ``fetch(dim)`` returns: the finite pairs and infinite
        classes of dimension ``dim``; the list of dimension 2 also holds the
        infinite classes of dimension 3 (only without the virtual maximum)."""
        p, e = self.counts()
        return p[dim] + e[dim] + (e[3] if dim == 2 else 0)

    def fetch(self, dim: int, out: np.ndarray | None = None) -> np.ndarray:
        """Pairs of dimension ``dim`` as a structured array of PAIR_DTYPE.
        ``out``: a host array of PAIR_DTYPE to copy into (e.g. a view of
        pinned memory, reused across calls); the result is its first part."""
        n = self.list_rows(dim)
        if out is None:
            out = np.empty(n, PAIR_DTYPE)
        elif out.dtype != PAIR_DTYPE or not out.flags.c_contiguous:
            raise ValueError("out must be a contiguous PAIR_DTYPE array")
        w = ctypes.c_int64(0)
        _check(self._lib.dms_fetch_pairs(self._h, dim, out.ctypes.data if n else None,
                                         len(out), ctypes.byref(w), 0), "dms_fetch_pairs")
        return out[: w.value]

    def fetch_device(self, dim: int, out_ptr: int, cap: int) -> int:
        w = ctypes.c_int64(0)
        _check(self._lib.dms_fetch_pairs(self._h, dim, ctypes.c_void_p(out_ptr), cap,
                                         ctypes.byref(w), 1), "dms_fetch_pairs")
        return w.value

    def stage_ms(self):
        ms = (ctypes.c_float * 8)()
        _check(self._lib.dms_get_stage_ms(self._h, ms), "dms_get_stage_ms")
        names = ("gradient", "sort", "d0", "d2", "d1", "output", "total", "h2d")
        return dict(zip(names, [float(x) for x in ms]))

    KERNELS = ("classify", "compact", "sort", "process_lower_stars", "emit", "d0_arcs",
               "d0_rounds", "d2_arcs", "d2_rounds", "d1_trace", "d1_reduce", "output")

    def kernel_ms(self):
        ms = (ctypes.c_float * 12)()
        _check(self._lib.dms_get_kernel_ms(self._h, ms), "dms_get_kernel_ms")
        return dict(zip(self.KERNELS, [float(x) for x in ms]))

    def work(self):
        """Work counts of the last compute (``dms_get_work``): edges the D1
        trace toggled and expanded, the longest chain of column additions."""
        w = (ctypes.c_int64 * 4)()
        _check(self._lib.dms_get_work(self._h, w), "dms_get_work")
        return {"trace_toggles": int(w[0]), "trace_expansions": int(w[1]),
                "d1_longest_chain": int(w[2])}

    def device_bytes(self) -> int:
        """Device memory this handle holds now (its arenas only grow)."""
        b = ctypes.c_int64(0)
        _check(self._lib.dms_get_device_bytes(self._h, ctypes.byref(b)), "dms_get_device_bytes")
        return int(b.value)

    def generators(self) -> dict:
        """{(birth edge id, death triangle id): array of the cycle's edge ids}
        for the D1 pairs of the last compute (a grid made with
        ``generators=True``; Sec. 8)."""
        w = ctypes.c_int64(0)
        st = self._lib.dms_fetch_generators(self._h, None, 0, ctypes.byref(w))
        if st not in (0, 7):
            _check(st, "dms_fetch_generators")
        buf = np.zeros(max(w.value, 1), np.int64)
        _check(self._lib.dms_fetch_generators(self._h, buf.ctypes.data, len(buf),
                                              ctypes.byref(w)), "dms_fetch_generators")
        out, i, flat = {}, 0, buf[: w.value]
        while i < len(flat):
            k = int(flat[i + 2])
            out[(int(flat[i]), int(flat[i + 1]))] = flat[i + 3:i + 3 + k].copy()
            i += 3 + k
        return out

    def result_id(self) -> int:
        """Identifier of the last successful compute (new for every compute)."""
        r = ctypes.c_uint64(0)
        _check(self._lib.dms_get_result_id(self._h, ctypes.byref(r)), "dms_get_result_id")
        return int(r.value)

    def stats(self):
        s = (ctypes.c_int64 * 16)()
        _check(self._lib.dms_get_stats(self._h, s), "dms_get_stats")
        names = ("critical_vertices", "c0", "c1", "c2", "c3", "launches", "levels_d0",
                 "levels_d2", "rounds_d1", "d1_columns", "d1_trace_overflow", "d1_additions",
                 "d1_pool_used", "d1_pool_grows", "d1_bytes_read", "d1_bytes_written")
        return dict(zip(names, [int(x) for x in s]))


class Batch(Grid):
    """A handle of ``dms_batch_create``: many fields of their own shapes, computed
    in one pass of the pipeline.  ``compute`` takes the fields one after another
    (a list of arrays/tensors indexed [z, y, x], or one packed array);
    ``fetch_fields(dim)`` returns one PAIR_DTYPE array per field, with ids
    relative to the field, equal to what a single-grid compute of that field
    returns."""

    def __init__(self, shapes_xyz, dtype, max_iters: int = 0, d1_mode: int = 0,
                 virtual_max: bool = True):
        self._lib = load()
        self.shapes_xyz = [tuple(int(s) for s in sh) for sh in shapes_xyz]
        self.dtype = np.dtype(dtype)
        if self.dtype not in _DTYPE_CODE:
            raise TypeError(f"unsupported dtype {self.dtype}")
        nf = len(self.shapes_xyz)
        flat = (ctypes.c_int64 * (3 * nf))(*[v for sh in self.shapes_xyz for v in sh])
        opts = _Options(int(bool(virtual_max)), int(max_iters), int(d1_mode))
        h = ctypes.c_void_p()
        _check(self._lib.dms_batch_create(nf, flat, _DTYPE_CODE[self.dtype], ctypes.byref(opts),
                                          ctypes.byref(h)), "dms_batch_create")
        self._h = h
        self.sizes = [a * b * c for a, b, c in self.shapes_xyz]
        self.n = int(sum(self.sizes))

    def reshape(self, shapes_xyz):
        """Re-targets this handle (and its device buffers) to another batch of
        field shapes (a list of (nx, ny, nz))."""
        if not shapes_xyz or not isinstance(shapes_xyz[0], (tuple, list)):
            raise DmsError(1, "a batch is reshaped to a list of field shapes")
        shapes = [tuple(int(s) for s in sh) for sh in shapes_xyz]
        flat = (ctypes.c_int64 * (3 * len(shapes)))(*[v for sh in shapes for v in sh])
        _check(self._lib.dms_batch_reshape(self._h, len(shapes), flat), "dms_batch_reshape")
        self.shapes_xyz = shapes
        self.sizes = [a * b * c for a, b, c in shapes]
        self.n = int(sum(self.sizes))
        return self

    def _field_ptr(self, values):
        if isinstance(values, (list, tuple)):
            try:
                import torch
            except ImportError:  # pragma: no cover
                torch = None
            if torch is not None and all(isinstance(v, torch.Tensor) for v in values):
                values = torch.cat([v.reshape(-1) for v in values])
            else:
                values = np.concatenate([np.asarray(v).reshape(-1) for v in values])
        try:
            import torch
        except ImportError:  # pragma: no cover
            torch = None
        if torch is not None and isinstance(values, torch.Tensor):
            if values.numel() != self.n or not values.is_contiguous():
                raise ValueError("the packed fields must be contiguous with sum(sizes) elements")
            if np.dtype(str(values.dtype).replace("torch.", "")) != self.dtype:
                raise TypeError("dtype mismatch")
            return values.data_ptr(), (0 if values.is_cuda else 1), values
        arr = np.ascontiguousarray(values).reshape(-1)
        if arr.size != self.n or arr.dtype != self.dtype:
            raise ValueError("packed size or dtype mismatch")
        return arr.ctypes.data, 1, arr

    def offsets(self, dim: int) -> np.ndarray:
        off = (ctypes.c_int64 * (len(self.shapes_xyz) + 1))()
        _check(self._lib.dms_batch_offsets(self._h, dim, off), "dms_batch_offsets")
        return np.array(off, dtype=np.int64)

    def fetch_fields(self, dim: int):
        allp = self.fetch(dim)
        off = self.offsets(dim)
        return [allp[off[f]:off[f + 1]] for f in range(len(self.shapes_xyz))]

    def results(self):
        """Per field: {dim: PAIR_DTYPE array}."""
        per = [self.fetch_fields(d) for d in range(3)]
        return [{d: per[d][f] for d in range(3)} for f in range(len(self.shapes_xyz))]


def classify_static(values, flags_out, critical_out, stream=None) -> int:
    """Binding of ``dms_classify_static`` (allocates nothing on the device).

    ``values``: CUDA tensor indexed [z, y, x]; ``flags_out``: CUDA uint8
    tensor of values.numel() bytes; ``critical_out``: CUDA int32 tensor whose
    length is the capacity.  Returns the number of PL-critical vertices."""
    import torch
    lib = load()
    nz, ny, nx = values.shape
    dt = np.dtype(str(values.dtype).replace("torch.", ""))
    n = ctypes.c_int64(0)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    _check(lib.dms_classify_static(ctypes.c_void_p(values.data_ptr()), _DTYPE_CODE[dt], nx, ny,
                                   nz, ctypes.c_void_p(flags_out.data_ptr()),
                                   ctypes.c_void_p(critical_out.data_ptr()),
                                   critical_out.numel(), ctypes.byref(n),
                                   ctypes.c_void_p(int(stream))), "dms_classify_static")
    return n.value


def diagram(values, shape_xyz=None, stream=None) -> dict:
    """D0, D1, D2 of a field (indexed [z, y, x]) as ``{dim: PAIR_DTYPE array}``."""
    if shape_xyz is None:
        nz, ny, nx = values.shape
        shape_xyz = (nx, ny, nz)
    dt = np.dtype(str(values.dtype).replace("torch.", "")) if not isinstance(values, np.ndarray) \
        else values.dtype
    with Grid(shape_xyz, dt) as g:
        g.compute(values, stream)
        return {d: g.fetch(d) for d in range(3)}
