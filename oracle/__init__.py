"""The oracle: a plain, slow CPU persistence pairing written from the paper.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  It
shares no code with the CUDA path (``paper_2206_13932_gb300``) and neither
imports the other.

Functions (all CPU, all exact):

- :func:`pairsimplices` -- Alg. 1 (PairSimplices) as the standard
  boundary-matrix reduction of the lexicographic filtration (Sec. 2.2,
  Sec. 2.4-2.5), keeping the pairs whose simplices have different maximum
  vertices plus the infinite-persistence classes (Sec. 4.1 (c), Sec. 6).
- :func:`fastpairs` -- the same standard reduction with result-preserving
  shortcuts (``fastpairs.c``): one dimension at a time from tets down to
  edges with clearing (Sec. 4, observation (a)), columns that need no
  addition regenerated from their ids instead of stored, and the filtration
  streamed lower star by lower star instead of sorted globally.  It reaches
  128^3 grids and more; the tests pin it equal to :func:`pairsimplices`.
- :func:`kruskal_d0` -- D0 by union-find over all edges (Sec. 1.1, the
  Edelsbrunner sub-level-set method), elder rule.
- :func:`kruskal_d2` -- D2 by union-find on the dual graph with a virtual
  maximum on the outer boundary (Sec. 5.2).
- :func:`sandwich` -- the method's own steps (``sandwich.c``): discrete
  gradient (Alg. 2), D0 and D2 by v-paths and union-find (Sec. 5), D1 by
  Alg. 3 with homologous propagation, with or without the virtual maximum
  (Sec. 5.2, App. A), and the 1-cycle generators of the D1 pairs (Sec. 8).
- :func:`gradient` -- the discrete gradient of that first step.
- :func:`simplex_counts`, :func:`simplex_vertices` -- the id scheme.

Parity of every function here is pinned by tests in ``tests/test_oracle_*.py``
(brute-force rank formulas, persistent Betti numbers, invariants, worked
fields).  :func:`sandwich` with the virtual maximum must equal
:func:`pairsimplices`; its generators are checked against the definition of a
cycle homologous to the boundary of the death triangle.  Without the virtual
maximum it is pinned only in part (invariants and the cases where it must
agree with the default); that part is marked "parity partly pinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, f) for f in ("pairsimplices.c", "sandwich.c", "fastpairs.c",
                                          "complex.h")]
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

DTYPES = {np.dtype(np.uint16): 0, np.dtype(np.float32): 1, np.dtype(np.float64): 2}
ERRORS = {1: "invalid argument", 2: "NaN in input", 3: "out of memory",
          4: "internal inconsistency"}
# result columns
COLS = ("dim", "birth", "death", "birth_vertex", "death_vertex", "essential",
        "birth_pos", "death_pos")


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(f) for f in _SRCS)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-Wall",
                               "-o", tmp] + [f for f in _SRCS if f.endswith(".c")])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            p64 = ctypes.POINTER(ctypes.c_int64)
            pp64 = ctypes.POINTER(p64)
            for name in ("oracle_kruskal_d0", "oracle_kruskal_d2"):
                f = getattr(lib, name)
                f.argtypes = [ctypes.c_int64] * 3 + [ctypes.c_int, ctypes.c_void_p, pp64, p64]
                f.restype = ctypes.c_int
            lib.oracle_pairsimplices.argtypes = ([ctypes.c_int64] * 3 +
                                                 [ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                                  pp64, p64])
            lib.oracle_pairsimplices.restype = ctypes.c_int
            lib.oracle_fastpairs.argtypes = ([ctypes.c_int64] * 3 +
                                             [ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                              pp64, p64, p64])
            lib.oracle_fastpairs.restype = ctypes.c_int
            lib.oracle_sandwich.argtypes = ([ctypes.c_int64] * 3 +
                                            [ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                             pp64, p64, pp64, p64])
            lib.oracle_sandwich.restype = ctypes.c_int
            lib.oracle_gradient.argtypes = [ctypes.c_int64] * 3 + [ctypes.c_int,
                                                                   ctypes.c_void_p, pp64, p64]
            lib.oracle_gradient.restype = ctypes.c_int
            lib.oracle_simplex_counts.argtypes = [ctypes.c_int64] * 3 + [p64]
            lib.oracle_simplex_counts.restype = ctypes.c_int
            lib.oracle_simplex_vertices.argtypes = [ctypes.c_int64] * 3 + [ctypes.c_int,
                                                                          ctypes.c_int64, p64]
            lib.oracle_simplex_vertices.restype = ctypes.c_int
            lib.oracle_free.argtypes = [ctypes.c_void_p]
            _lib = lib
    return _lib


def _field(values: np.ndarray):
    """(nx, ny, nz, dtype code, contiguous array) for a field indexed [z, y, x]."""
    values = np.ascontiguousarray(values)
    if values.ndim != 3:
        raise ValueError("field must be 3D, indexed [z, y, x] (x fastest)")
    if values.dtype not in DTYPES:
        raise TypeError(f"unsupported dtype {values.dtype}")
    nz, ny, nx = values.shape
    return nx, ny, nz, DTYPES[values.dtype], values


def _call(fn, values, *extra, tail=()):
    nx, ny, nz, code, arr = _field(values)
    out = ctypes.POINTER(ctypes.c_int64)()
    n = ctypes.c_int64(0)
    st = fn(nx, ny, nz, code, arr.ctypes.data_as(ctypes.c_void_p), *extra,
            ctypes.byref(out), ctypes.byref(n), *tail)
    if st:
        raise ValueError(f"oracle: {ERRORS.get(st, st)}")
    try:
        rows = np.ctypeslib.as_array(out, shape=(n.value, 8)).copy() if n.value else \
            np.zeros((0, 8), np.int64)
    finally:
        _load().oracle_free(out)
    return rows


def pairsimplices(values: np.ndarray, keep_zero: bool = False) -> np.ndarray:
    """Standard reduction of the whole lexicographic filtration.

    Returns an ``(n, 8)`` int64 array with the columns of :data:`COLS`.
    Zero-persistence pairs (same maximum vertex) are dropped unless
    ``keep_zero``.
    """
    lib = _load()
    return _call(lib.oracle_pairsimplices, values, int(bool(keep_zero)))


def fastpairs(values: np.ndarray, keep_zero: bool = False, stats: dict | None = None) -> np.ndarray:
    """The pairs of :func:`pairsimplices`, computed by the fast-mode standard
    reduction (``fastpairs.c``).  The two filtration-position columns are -1.
    ``stats``: if given, receives ``additions`` (column additions made)."""
    lib = _load()
    adds = ctypes.c_int64(0)
    rows = _call(lib.oracle_fastpairs, values, int(bool(keep_zero)), tail=(ctypes.byref(adds),))
    if stats is not None:
        stats["additions"] = int(adds.value)
    return rows


def kruskal_d0(values: np.ndarray) -> np.ndarray:
    """D0 (plus the essential class of the global minimum) by union-find."""
    return _call(_load().oracle_kruskal_d0, values)


def kruskal_d2(values: np.ndarray) -> np.ndarray:
    """D2 by union-find on the dual graph with a virtual maximum."""
    return _call(_load().oracle_kruskal_d2, values)


def _take(ptr, n, width):
    try:
        if n == 0:
            return np.zeros((0, width) if width else 0, np.int64)
        shape = (n, width) if width else (n,)
        return np.ctypeslib.as_array(ptr, shape=shape).copy()
    finally:
        _load().oracle_free(ptr)


def sandwich(values: np.ndarray, virtual_max: bool = True):
    """The diagrams by the method's own steps (``sandwich.c``).

    Returns ``(rows, generators)``: ``rows`` as :func:`pairsimplices` (columns
    :data:`COLS`, infinite classes flagged), and ``generators`` a dict
    ``{(birth_edge_id, death_triangle_id): [edge ids]}`` holding, for every D1
    pair, the cycle on which the homologous propagation of Alg. 3 stopped,
    in increasing filtration order.
    """
    lib = _load()
    nx, ny, nz, code, arr = _field(values)
    rows_p = ctypes.POINTER(ctypes.c_int64)()
    gen_p = ctypes.POINTER(ctypes.c_int64)()
    n_rows, n_gen = ctypes.c_int64(0), ctypes.c_int64(0)
    st = lib.oracle_sandwich(nx, ny, nz, code, arr.ctypes.data_as(ctypes.c_void_p),
                             int(bool(virtual_max)), ctypes.byref(rows_p),
                             ctypes.byref(n_rows), ctypes.byref(gen_p), ctypes.byref(n_gen))
    if st:
        raise ValueError(f"oracle: {ERRORS.get(st, st)}")
    rows = _take(rows_p, n_rows.value, 8)
    flat = _take(gen_p, n_gen.value, 0)
    gens, i = {}, 0
    while i < len(flat):
        k = int(flat[i + 2])
        gens[(int(flat[i]), int(flat[i + 1]))] = [int(e) for e in flat[i + 3:i + 3 + k]]
        i += 3 + k
    return rows, gens


def gradient(values: np.ndarray) -> np.ndarray:
    """The discrete gradient of Alg. 2: one ``(dim, id, partner_dim,
    partner_id)`` row per simplex in lexicographic order (``-1, -1`` for a
    critical simplex)."""
    return _call4(_load().oracle_gradient, values)


def _call4(fn, values):
    nx, ny, nz, code, arr = _field(values)
    out = ctypes.POINTER(ctypes.c_int64)()
    n = ctypes.c_int64(0)
    st = fn(nx, ny, nz, code, arr.ctypes.data_as(ctypes.c_void_p), ctypes.byref(out),
            ctypes.byref(n))
    if st:
        raise ValueError(f"oracle: {ERRORS.get(st, st)}")
    return _take(out, n.value, 4)


def simplex_counts(nx: int, ny: int, nz: int) -> tuple:
    c = (ctypes.c_int64 * 4)()
    if _load().oracle_simplex_counts(nx, ny, nz, c):
        raise ValueError("bad grid")
    return tuple(c)


def simplex_vertices(shape_xyz, dim: int, sid: int):
    """Vertex ids of simplex ``sid`` of dimension ``dim``, or None if invalid."""
    nx, ny, nz = shape_xyz
    vs = (ctypes.c_int64 * 4)()
    if not _load().oracle_simplex_vertices(nx, ny, nz, dim, sid, vs):
        return None
    return tuple(vs[: dim + 1])


def diagram(values: np.ndarray) -> dict:
    """Oracle diagram as ``{dim: set of (birth_id, death_id)}`` plus
    ``'essential'``: set of (dim, birth_id)."""
    rows = pairsimplices(values)
    out = {0: set(), 1: set(), 2: set(), "essential": set()}
    for r in rows:
        if r[5]:
            out["essential"].add((int(r[0]), int(r[1])))
        else:
            out[int(r[0])].add((int(r[1]), int(r[2])))
    return out
