"""Continuous-batching diagram server.

Requests (one scalar field each, any shape) are admitted as soon as a slot
and enough of the device-memory budget are free; a request that arrives
while others are on the GPU starts right away in a free slot, so the work of
several requests overlaps on the device.  Each slot is a host thread that
owns a CUDA stream and one reusable ``dms_grid`` per dtype (reshaped per
request, so its device buffers are kept across requests); the C ABI calls
release the GIL, so slots drive the GPU concurrently.  With max_batch > 1 and
a backlog (more requests waiting than ``batch_above``, by default the number
of slots) a slot takes every waiting request it can (up to max_batch, within
the budget) and runs them as one batch -- one pass of the pipeline over the
disjoint union of their grids -- on a reusable batch handle.  Without a
backlog requests run one by one: a batch raises the throughput of a saturated
server, but a request in it waits for the whole batch.  Each result is the same as the
request's diagram computed alone (the pipeline is deterministic, handles
share no state, and a batch's per-field pairs equal the single-grid ones).

Device memory: the requests in flight stay within ``mem_budget``, each
charged by the estimate ``request_bytes``.  A handle's buffers only grow, so a
slot keeps at most one handle of each kind (grid, batch) between requests,
and only while the device memory they really hold (``device_bytes``, which
includes D1 pools grown on noisy fields; the request's estimate for the one
just used) fits the slot's share of the budget (``keeps_buffers``); above it
the other kind's handle is freed first, then the one just used.  A slot's idle
handles therefore hold at most ``mem_budget / slots``, measured, not
estimated.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import Batch, Grid


def request_bytes(n_vertices: int, itemsize: int) -> int:
    """Device bytes one request may hold: its field, the per-vertex state
    (flags, ranks, 48-byte gradient records) and a bound for the critical
    simplices, arcs and D1 columns."""
    return int(n_vertices) * (itemsize + 1 + 4 + 48 + 96)


def keeps_buffers(need: int, budget: int, slots: int) -> bool:
    """Whether a slot keeps a handle (and its device buffers) that holds
    ``need`` bytes: only within the slot's share of the budget."""
    return need <= budget // max(1, int(slots))


def select_batch(pending, in_flight: int, budget: int, max_batch: int,
                 max_vertices: int | None = None, batch_above: int | None = None):
    """Admission: how many of the pending requests (a list of (vertices,
    dtype) in arrival order) start now, and their bytes.  The oldest ones that
    fit the free budget, up to max_batch and (after the first) up to
    max_vertices in all, all of the head's dtype; nothing overtakes a head
    request that does not fit, so it is never starved.  The vertex bound keeps
    one batched pass short, so requests behind it wait less.  With
    ``batch_above`` set, only a backlog of more than that many pending
    requests is batched; a shorter queue is served one request at a time."""
    if batch_above is not None and len(pending) <= batch_above:
        max_batch = 1
    k, need, verts = 0, 0, 0
    for size, dtype in pending:
        dt = np.dtype(dtype)
        if k and dt != np.dtype(pending[0][1]):
            break
        if k and max_vertices is not None and verts + size > max_vertices:
            break
        r = request_bytes(size, dt.itemsize)
        if in_flight + need + r > budget:
            break
        k += 1
        need += r
        verts += size
        if k == max_batch:
            break
    return k, need


class CudaBackend:
    """What a slot needs from the device: a stream of its own, the context
    that makes it current, its handle for the C ABI, and the handle types."""

    def __init__(self):
        import torch
        self.torch = torch
        self.Grid, self.Batch = Grid, Batch

    def stream(self):
        return self.torch.cuda.Stream()

    def current(self, stream):
        return self.torch.cuda.stream(stream)

    @staticmethod
    def handle(stream):
        return stream.cuda_stream


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
    """``slots`` concurrent passes at most, within ``mem_budget`` bytes.  With
    ``max_batch`` > 1, while more than ``batch_above`` requests wait (default:
    the number of slots), a free slot takes up to max_batch of them (in
    arrival order, one dtype, within the budget, and after the first at most
    ``max_batch_vertices`` vertices in all) and computes them as one batch
    (``dms_batch_create``): one pass of the pipeline for all of them."""

    def __init__(self, slots: int = 4, mem_budget: int = 16 << 30, max_batch: int = 1,
                 backend=None, max_batch_vertices: int | None = None,
                 batch_above: int | None = None):
        self._be = backend if backend is not None else CudaBackend()
        self.slots = slots
        self.mem_budget = mem_budget
        self.max_batch = max(1, int(max_batch))
        self.max_batch_vertices = max_batch_vertices
        self.batch_above = slots if batch_above is None else int(batch_above)
        self._pending = []                 # FIFO of admitted-later requests
        self._cv = threading.Condition()
        self._in_flight_bytes = 0
        self._stop = False
        self._workers = []
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
        """The next batch to run (see select_batch), waiting until one fits."""
        with self._cv:
            while True:
                if self._stop and not self._pending:
                    return None
                k, need = select_batch([(r.values.size, r.values.dtype) for r in self._pending],
                                       self._in_flight_bytes, self.mem_budget, self.max_batch,
                                       self.max_batch_vertices, self.batch_above)
                if k:
                    take = self._pending[:k]
                    del self._pending[:k]
                    self._in_flight_bytes += need
                    return take, need
                self._cv.wait(0.05)

    def _release(self, need):
        with self._cv:
            self._in_flight_bytes -= need
            self._cv.notify_all()

    def _worker(self, k: int):
        be = self._be
        try:
            stream, setup_error = be.stream(), None
        except Exception as e:   # every request this slot takes then reports it
            stream, setup_error = None, e
        held = {}            # kind -> (dtype, handle): at most one of each kind between requests
        while True:
            got = self._take()
            if got is None:
                break
            reqs, need = got
            t = time.perf_counter()
            for r in reqs:
                r.admitted = t
            kind = "grid" if len(reqs) == 1 else "batch"
            try:
                if setup_error is not None:
                    raise setup_error
                dt = reqs[0].values.dtype
                shapes = [(r.values.shape[2], r.values.shape[1], r.values.shape[0]) for r in reqs]
                h = None
                if kind in held and held[kind][0] == dt:
                    h = held[kind][1]
                elif kind in held:                  # another dtype: free it first
                    held.pop(kind)[1].close()
                with be.current(stream):
                    if kind == "grid":
                        if h is None:
                            h = be.Grid(shapes[0], dt)
                        elif h.shape_xyz != shapes[0]:
                            h.reshape(shapes[0])
                        held[kind] = (dt, h)
                        h.compute(reqs[0].values, stream=be.handle(stream))
                        reqs[0].result = {d: h.fetch(d) for d in range(3)}
                    else:
                        if h is None:
                            h = be.Batch(shapes, dt)
                        else:
                            h.reshape(shapes)
                        held[kind] = (dt, h)
                        h.compute([r.values for r in reqs], stream=be.handle(stream))
                        for r, res in zip(reqs, h.results()):
                            r.result = res
            except Exception as e:   # reported to the caller
                for r in reqs:
                    r.error = e
            self._trim(held, kind, need)
            t = time.perf_counter()
            self._release(need)
            for r in reqs:
                r.finished = t
                r.done.set()
        for _, h in held.values():
            h.close()

    def _trim(self, held, used, need):
        """Frees held handles until what they hold fits the slot's share:
        the kind not just used first."""
        def size(kind):
            try:
                b = held[kind][1].device_bytes()
            except Exception:
                return None
            return max(need, b) if kind == used else b
        for kind in sorted(held, key=lambda k: k == used):
            sizes = [size(k) for k in held]
            if None not in sizes and keeps_buffers(sum(sizes), self.mem_budget, self.slots):
                return
            held.pop(kind)[1].close()


def run_stream(fields, arrivals, slots: int, mem_budget: int = 16 << 30, max_batch: int = 1,
               backend=None, **server_options):
    """Replays requests arriving at ``arrivals`` (seconds from start) through
    a server; returns the requests (with timings and results) and the wall
    time.  ``server_options`` go to DiagramServer (max_batch_vertices,
    batch_above)."""
    srv = DiagramServer(slots=slots, mem_budget=mem_budget, max_batch=max_batch,
                        backend=backend, **server_options)
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
    """Latency percentiles (arrival to result), split into the wait for a slot
    (arrival to admission) and the service (admission to result)."""
    lat = np.array([r.finished - r.arrival for r in reqs]) * 1e3
    wait = np.array([r.admitted - r.arrival for r in reqs]) * 1e3
    serv = np.array([r.finished - r.admitted for r in reqs]) * 1e3
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()),
            "wait_p50_ms": float(np.percentile(wait, 50)),
            "wait_p99_ms": float(np.percentile(wait, 99)),
            "service_p50_ms": float(np.percentile(serv, 50)),
            "service_p99_ms": float(np.percentile(serv, 99))}
