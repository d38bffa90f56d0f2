"""Autotuner of the launch shapes and capacities of a handle.

The tunables (``dms_set_tuning``, in ``TUNABLES`` order) change only how fast
a diagram is computed, never the diagram: thread-block sizes of
ProcessLowerStars and of the first D1 trace pass, the number of trace
threads per SM and their heap size, the number of active columns below which
a whole block performs a column's additions (and the asynchronous tail
starts), the heap size of a lazy advance, the column density below which D1
mode 0 reduces lazily, whether the tail of the traced reduction runs as
one asynchronous pass, when ProcessLowerStars sorts its stars by shape, and
whether D2's ascending walks run on a second stream beside D0.

``tune`` runs a coordinate descent: starting from the handle's current
values, it tries each candidate of one tunable with the others fixed, keeps
a candidate that is faster by more than ``min_gain`` (median device time of
``repeats`` computes), and moves to the next tunable.  Results can be kept in
a JSON cache keyed by dtype, size class and D1 mode (``save``/``load``).
"""
from __future__ import annotations

import ctypes
import json
import os
import time

import numpy as np

from . import _check

TUNABLES = ("pls_block", "trace_block", "trace_per_sm", "trace_heap", "red_block_below",
            "lazy_heap", "lazy_density", "red_async", "pls_sort", "d2_beside_d0")
DEFAULT = (128, 128, 2048, 48, -1, 48, 32, 1, 1, 1)
CANDIDATES = {
    "pls_block": (64, 128, 256),
    "trace_block": (64, 128, 256),
    "trace_per_sm": (1024, 2048, 4096),
    "trace_heap": (32, 48, 96),
    "red_block_below": (-1, 4096, 16384),
    "lazy_heap": (32, 48, 96),
    "lazy_density": (16, 32, 64),
    "red_async": (0, 1),
    "pls_sort": (0, 1, 2),
    "d2_beside_d0": (0, 1),
}


def get_tuning(grid) -> tuple:
    v = (ctypes.c_int32 * len(TUNABLES))()
    _check(grid._lib.dms_get_tuning(grid._h, v, len(TUNABLES)), "dms_get_tuning")
    return tuple(int(x) for x in v)


def set_tuning(grid, values) -> None:
    v = (ctypes.c_int32 * len(TUNABLES))(*[int(x) for x in values])
    _check(grid._lib.dms_set_tuning(grid._h, v, len(TUNABLES)), "dms_set_tuning")


def valid(values) -> bool:
    """The ranges ``dms_set_tuning`` accepts (it refuses anything else)."""
    if len(values) != len(TUNABLES):
        return False
    d = dict(zip(TUNABLES, (int(x) for x in values)))

    def block(b, most):
        return 32 <= b <= most and b % 32 == 0
    return (block(d["pls_block"], 512) and block(d["trace_block"], 256) and
            d["trace_block"] <= d["trace_per_sm"] <= 8192 and
            d["trace_per_sm"] % d["trace_block"] == 0 and
            8 <= d["trace_heap"] <= 1024 and d["red_block_below"] >= -1 and
            8 <= d["lazy_heap"] <= 1024 and 1 <= d["lazy_density"] <= 4096 and
            d["red_async"] in (0, 1) and d["pls_sort"] in (0, 1, 2) and
            d["d2_beside_d0"] in (0, 1))


def measure(grid, field, repeats: int = 3) -> float:
    """Median device milliseconds of ``repeats`` computes of ``field``."""
    ts = []
    for _ in range(repeats):
        grid.compute(field)
        ts.append(grid.stage_ms()["total"])
    return float(np.median(ts))


def tune(grid, field, repeats: int = 3, min_gain: float = 0.02, budget_s: float | None = None):
    """Coordinate descent over CANDIDATES on ``grid`` computing ``field``.
    Returns (best values, {"start_ms", "best_ms", "trials": [(values, ms)],
    "seconds"}).  The handle is left set to the best values."""
    t0 = time.perf_counter()
    grid.compute(field)                         # warm-up: buffers sized, tables loaded
    cur = get_tuning(grid)
    best = measure(grid, field, repeats)
    trials = [(cur, best)]
    start_ms = best
    for k, name in enumerate(TUNABLES):
        for cand in CANDIDATES[name]:
            if budget_s is not None and time.perf_counter() - t0 > budget_s:
                break
            if cand == cur[k]:
                continue
            vals = tuple(cand if i == k else x for i, x in enumerate(cur))
            if not valid(vals):
                continue
            set_tuning(grid, vals)
            t = measure(grid, field, repeats)
            trials.append((vals, t))
            if t < best * (1.0 - min_gain):
                best, cur = t, vals
        set_tuning(grid, cur)
    return cur, {"start_ms": start_ms, "best_ms": best, "trials": trials,
                 "seconds": time.perf_counter() - t0}


def cache_key(dtype, n_vertices: int, d1_mode: int = 0) -> str:
    return f"{np.dtype(dtype).name}:2^{int(np.log2(max(n_vertices, 1)))}:mode{d1_mode}"


def load(path: str, key: str):
    if not os.path.exists(path):
        return None
    with open(path) as f:
        v = json.load(f).get(key)
    return tuple(v) if v else None


def save(path: str, key: str, values) -> None:
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    data[key] = list(values)
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
