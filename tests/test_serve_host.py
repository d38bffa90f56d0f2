"""The diagram server's host logic with a fake device backend (no GPU).

The fake handles stand in for ``Grid`` and ``Batch``: a "diagram" is the sum
of the field's values, so every request can be matched to its own result.
Checked: every request completes with its own result, alone or in batches;
the bytes of the requests computing at once never exceed the budget; a
handle is kept after a request within the slot's share of the budget and
freed after a larger one; an error of the compute call (a fake of the
failing C call) reaches that request only, and the server goes on.
"""
import contextlib
import threading
import time

import numpy as np
import pytest

from paper_2206_13932_gb300 import DmsError
from paper_2206_13932_gb300 import serve


class _Ledger:
    def __init__(self):
        self.lock = threading.Lock()
        self.now = 0
        self.peak = 0
        self.created = 0
        self.closed = 0

    def enter(self, nbytes):
        with self.lock:
            self.now += nbytes
            self.peak = max(self.peak, self.now)

    def leave(self, nbytes):
        with self.lock:
            self.now -= nbytes

    def count(self, name):
        with self.lock:
            setattr(self, name, getattr(self, name) + 1)


def _bytes(v):
    return serve.request_bytes(v.size, v.dtype.itemsize)


def _diagram(v):
    if np.isnan(v).any():
        raise DmsError(2, "dms_compute_diagram")    # DMS_ERR_NAN, as the library reports it
    return {d: np.array([float(v.sum()), d]) for d in range(3)}


class _FakeGrid:
    ledger = None
    extra = 0          # device bytes a handle holds beyond the request's estimate

    def __init__(self, shape_xyz, dtype):
        self.shape_xyz = tuple(shape_xyz)
        self.dtype = np.dtype(dtype)
        self.ledger.count("created")
        self.res = None
        self.nbytes = 0

    def device_bytes(self):
        return self.nbytes

    def reshape(self, shape_xyz):
        self.shape_xyz = tuple(shape_xyz)
        return self

    def compute(self, values, stream=None):
        self.ledger.enter(_bytes(values))
        self.nbytes = max(self.nbytes, _bytes(values) + self.extra)   # buffers only grow
        try:
            time.sleep(0.002)
            self.res = _diagram(values)
        finally:
            self.ledger.leave(_bytes(values))

    def fetch(self, d):
        return self.res[d]

    def close(self):
        self.ledger.count("closed")


class _FakeBatch(_FakeGrid):
    def __init__(self, shapes, dtype):
        super().__init__((0, 0, 0), dtype)
        self.shapes = list(shapes)

    def reshape(self, shapes):
        self.shapes = list(shapes)
        return self

    def compute(self, fields, stream=None):
        n = sum(_bytes(f) for f in fields)
        self.ledger.enter(n)
        self.nbytes = max(self.nbytes, n + self.extra)
        try:
            time.sleep(0.002)
            self.per = [_diagram(f) for f in fields]
        finally:
            self.ledger.leave(n)

    def results(self):
        return self.per


class _FakeBackend:
    def __init__(self, extra=0):
        self.ledger = _Ledger()
        grid = type("Grid", (_FakeGrid,), {"ledger": self.ledger, "extra": extra})
        batch = type("Batch", (_FakeBatch,), {"ledger": self.ledger, "extra": extra})
        self.Grid, self.Batch = grid, batch

    def stream(self):
        return object()

    def current(self, stream):
        return contextlib.nullcontext()

    @staticmethod
    def handle(stream):
        return 0


def _fields(n, seed=0, lo=4, hi=20):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nx, ny, nz = (int(x) for x in rng.integers(lo, hi, 3))
        out.append(rng.random((nz, ny, nx)).astype(np.float32))
    return out


@pytest.mark.parametrize("max_batch", [1, 8])
def test_every_request_gets_its_own_result_within_the_budget(max_batch):
    fields = _fields(60, seed=1)
    budget = 4 * max(_bytes(f) for f in fields)
    be = _FakeBackend()
    reqs, _ = serve.run_stream(fields, np.zeros(len(fields)), slots=4, mem_budget=budget,
                               max_batch=max_batch, backend=be)
    for r, f in zip(reqs, fields):
        assert r.error is None and r.result[0][0] == float(f.sum())
        assert r.finished >= r.admitted >= r.arrival
    assert 0 < be.ledger.peak <= budget
    assert be.ledger.created == be.ledger.closed      # every handle freed at shutdown


def test_handles_kept_within_the_share_and_freed_above_it():
    small = _fields(6, seed=2, lo=4, hi=6)
    budget = 2 * 10 * max(_bytes(f) for f in small)   # every request within its share
    be = _FakeBackend()
    serve.run_stream(small, np.zeros(len(small)), slots=2, mem_budget=budget, backend=be)
    assert be.ledger.created <= 2                      # one reused handle per slot at most
    big = np.ones((40, 40, 40), np.float32)
    budget = 2 * _bytes(big) - 1                      # the request exceeds its slot's share
    be = _FakeBackend()
    serve.run_stream([big] * 3, np.arange(3) * 0.05, slots=2, mem_budget=budget, backend=be)
    assert be.ledger.created == 3 and be.ledger.closed == 3   # freed after every request


def test_handles_holding_more_than_their_estimate_are_freed():
    """A handle whose real device memory (device_bytes: pools grown on noisy
    fields) exceeds the slot's share is freed after the request even though
    the request's estimate fit; each slot keeps one handle at most."""
    small = _fields(6, seed=3, lo=4, hi=6)
    budget = 2 * 10 * max(_bytes(f) for f in small)      # estimates within the share
    be = _FakeBackend(extra=budget)                      # but every handle holds more
    serve.run_stream(small, np.zeros(len(small)), slots=2, mem_budget=budget, backend=be)
    assert be.ledger.created == len(small) and be.ledger.closed == len(small)
    mixed = _fields(12, seed=6, lo=4, hi=6)
    mixed = [f if i % 2 else f.astype(np.float64) for i, f in enumerate(mixed)]
    be = _FakeBackend()
    serve.run_stream(mixed, np.arange(len(mixed)) * 0.01, slots=1,
                     mem_budget=10 * budget, backend=be)
    assert be.ledger.created == be.ledger.closed == len(mixed)   # dtype switch frees the other


def test_a_slot_keeps_one_handle_of_each_kind():
    """With batching on, a backlog runs as batches and the requests after it
    one by one; a slot keeps its batch handle and its grid handle (both
    within its share) instead of freeing one to make the other."""
    fields = _fields(40, seed=7, lo=4, hi=6)
    be = _FakeBackend()
    reqs, _ = serve.run_stream(fields, np.r_[np.zeros(30), 0.05 + 0.02 * np.arange(10)],
                               slots=2, mem_budget=10 ** 9, max_batch=8, backend=be)
    assert all(r.error is None for r in reqs)
    assert be.ledger.created <= 4 and be.ledger.created == be.ledger.closed


def test_a_failing_compute_reaches_only_its_request():
    fields = _fields(20, seed=4)
    fields[7] = fields[7].copy()
    fields[7].flat[3] = np.nan
    be = _FakeBackend()
    reqs, _ = serve.run_stream(fields, np.zeros(len(fields)), slots=3, backend=be)
    for i, (r, f) in enumerate(zip(reqs, fields)):
        if i == 7:
            assert isinstance(r.error, DmsError) and r.error.status == 2
        else:
            assert r.error is None and r.result[0][0] == float(f.sum())


def test_requests_larger_than_the_budget_are_refused():
    be = _FakeBackend()
    srv = serve.DiagramServer(slots=1, mem_budget=1000, backend=be)
    try:
        with pytest.raises(ValueError):
            srv.submit(serve.Request(arrival=0.0, req_id=0,
                                     values=np.zeros((8, 8, 8), np.float32)))
    finally:
        srv.close()


def test_a_slot_without_a_stream_fails_its_requests_instead_of_hanging():
    class NoStream(_FakeBackend):
        def stream(self):
            raise RuntimeError("no device")
    reqs, _ = serve.run_stream(_fields(5, seed=5), np.zeros(5), slots=2, backend=NoStream())
    assert all(isinstance(r.error, RuntimeError) for r in reqs)
