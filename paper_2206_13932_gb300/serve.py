"""Continuous-batching diagram server.

Requests (one scalar field each, any shape) are admitted as soon as a slot
and enough of the device-memory budget are free; a request that arrives
while others are on the GPU starts right away in a free slot, so the work of
several requests overlaps on the device.  Each slot is a host thread that
owns a CUDA stream and one reusable ``dms_grid`` per dtype (reshaped per
request, so its device buffers are kept across requests); the C ABI calls
release the GIL, so slots drive the GPU concurrently.  Each result is the
same as the request's diagram computed alone (the pipeline is deterministic
and handles share no state).
"""
from __future__ import annotations

import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import Grid


def request_bytes(n_vertices: int, itemsize: int) -> int:
    """Device bytes one request may hold: its field, the per-vertex state
    (flags, ranks, 48-byte gradient records) and a bound for the critical
    simplices, arcs and D1 columns."""
    return int(n_vertices) * (itemsize + 1 + 4 + 48 + 96)


@dataclass(order=True)
class Request:
    arrival: float
    req_id: int = field(compare=False)
    values: np.ndarray = field(compare=False, repr=False)
    done: threading.Event = field(default_factory=threading.Event, compare=False, repr=False)
    result: dict = field(default=None, compare=False, repr=False)
    error: Exception = field(default=None, compare=False, repr=False)
    admitted: float = field(default=0.0, compare=False)
    finished: float = field(default=0.0, compare=False)


class DiagramServer:
    """``slots`` concurrent requests at most, within ``mem_budget`` bytes."""

    def __init__(self, slots: int = 4, mem_budget: int = 16 << 30):
        import torch
        self.slots = slots
        self.mem_budget = mem_budget
        self._pending = []                 # FIFO of admitted-later requests
        self._cv = threading.Condition()
        self._in_flight_bytes = 0
        self._stop = False
        self._workers = []
        self._torch = torch
        for k in range(slots):
            t = threading.Thread(target=self._worker, args=(k,), daemon=True)
            t.start()
            self._workers.append(t)

    def submit(self, req: Request) -> Request:
        need = request_bytes(req.values.size, req.values.dtype.itemsize)
        if need > self.mem_budget:
            raise ValueError("request larger than the memory budget")
        with self._cv:
            self._pending.append(req)
            self._cv.notify_all()
        return req

    def close(self):
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        for t in self._workers:
            t.join()

    def _take(self):
        """The oldest pending request that fits the free budget (FIFO order;
        a large head request waits until enough memory is free)."""
        with self._cv:
            while True:
                if self._stop and not self._pending:
                    return None
                if self._pending:
                    req = self._pending[0]
                    need = request_bytes(req.values.size, req.values.dtype.itemsize)
                    if self._in_flight_bytes + need <= self.mem_budget:
                        self._pending.pop(0)
                        self._in_flight_bytes += need
                        return req, need
                self._cv.wait(0.05)

    def _release(self, need):
        with self._cv:
            self._in_flight_bytes -= need
            self._cv.notify_all()

    def _worker(self, k: int):
        torch = self._torch
        stream = torch.cuda.Stream()
        grids = {}
        while True:
            got = self._take()
            if got is None:
                break
            req, need = got
            req.admitted = time.perf_counter()
            try:
                v = req.values
                nz, ny, nx = v.shape
                g = grids.get(v.dtype)
                if g is None:
                    g = grids[v.dtype] = Grid((nx, ny, nz), v.dtype)
                elif g.shape_xyz != (nx, ny, nz):
                    g.reshape((nx, ny, nz))
                with torch.cuda.stream(stream):
                    g.compute(v, stream=stream.cuda_stream)
                    req.result = {d: g.fetch(d) for d in range(3)}
            except Exception as e:   # reported to the caller
                req.error = e
            req.finished = time.perf_counter()
            self._release(need)
            req.done.set()
        for g in grids.values():
            g.close()


def run_stream(fields, arrivals, slots: int, mem_budget: int = 16 << 30):
    """Replays requests arriving at ``arrivals`` (seconds from start) through
    a server; returns the requests (with timings and results) and the wall
    time."""
    srv = DiagramServer(slots=slots, mem_budget=mem_budget)
    reqs = []
    t0 = time.perf_counter()
    for i, (f, a) in enumerate(zip(fields, arrivals)):
        now = time.perf_counter() - t0
        if a > now:
            time.sleep(a - now)
        reqs.append(srv.submit(Request(arrival=t0 + a, req_id=i, values=f)))
    for r in reqs:
        r.done.wait()
    wall = time.perf_counter() - t0
    srv.close()
    return reqs, wall


def latency_stats(reqs):
    lat = np.array([r.finished - r.arrival for r in reqs]) * 1e3
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean())}
