"""Continuous-batching server: every result equals the request's diagram
computed alone (bit-exact, the pairing is integer work), while requests of
different shapes overlap on the GPU and are admitted under a memory budget."""
import numpy as np
import pytest

import synthfields as sf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dms():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2206_13932_gb300 as m
    m.build()
    return m


def _alone(dms, v):
    nz, ny, nx = v.shape
    with dms.Grid((nx, ny, nz), v.dtype) as g:
        g.compute(v)
        return {d: g.fetch(d) for d in range(3)}


def test_results_identical_alone_and_in_the_mix(dms):
    from paper_2206_13932_gb300 import serve
    fields = sf.serving_fields(24, seed0=4000, lo=8, hi=40)
    fields += [sf.white_noise(sh, 90 + i) for i, sh in enumerate(sf.serving_shapes(8, 91, 8, 40))]
    want = [_alone(dms, f) for f in fields]
    # all at once (maximal overlap), then staggered, with a budget that forces waiting
    for arrivals, budget in ((np.zeros(len(fields)), 1 << 34),
                             (sf.poisson_arrivals(len(fields), 400.0), 6 * serve.request_bytes(
                                 40 ** 3, 4))):
        reqs, wall = serve.run_stream(fields, arrivals, slots=4, mem_budget=budget)
        for r, w in zip(reqs, want):
            assert r.error is None
            for d in range(3):
                assert r.result[d].tobytes() == w[d].tobytes()
        stats = serve.latency_stats(reqs)
        assert stats["p99_ms"] >= stats["p50_ms"] > 0


def test_batched_slots_identical_alone(dms):
    from paper_2206_13932_gb300 import serve
    fields = sf.serving_fields(40, seed0=4100, lo=8, hi=40)
    fields += [sf.white_noise(sh, 190 + i) for i, sh in enumerate(sf.serving_shapes(8, 191, 8, 32))]
    want = [_alone(dms, f) for f in fields]
    for arrivals, budget in ((np.zeros(len(fields)), 1 << 34),
                             (sf.poisson_arrivals(len(fields), 600.0),
                              12 * serve.request_bytes(40 ** 3, 4))):
        reqs, _ = serve.run_stream(fields, arrivals, slots=3, mem_budget=budget, max_batch=8)
        for r, w in zip(reqs, want):
            assert r.error is None
            for d in range(3):
                assert r.result[d].tobytes() == w[d].tobytes()


def test_reshaped_handle_matches_fresh_handles(dms):
    fields = [sf.white_noise(sh, 7) for sh in ((9, 7, 5), (20, 11, 13), (6, 6, 6), (31, 2, 17))]
    with dms.Grid((4, 4, 4), np.float32) as g:
        for f in fields:
            nz, ny, nx = f.shape
            g.reshape((nx, ny, nz)).compute(f)
            got = {d: g.fetch(d) for d in range(3)}
            want = _alone(dms, f)
            for d in range(3):
                assert got[d].tobytes() == want[d].tobytes()
