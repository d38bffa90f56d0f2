"""Admission of the diagram server (host logic, no GPU): arrival order, the
memory budget, the batch cap and one dtype per batch."""
import numpy as np

from paper_2206_13932_gb300.serve import keeps_buffers, request_bytes, select_batch


def _req(n, dt=np.float32):
    return (n, np.dtype(dt))


def test_oldest_requests_within_budget_and_cap():
    pend = [_req(1000), _req(2000), _req(3000), _req(4000)]
    b = request_bytes(1000, 4) + request_bytes(2000, 4) + request_bytes(3000, 4)
    assert select_batch(pend, 0, b, 8) == (3, b)
    assert select_batch(pend, 0, 10 ** 12, 2) == (2, request_bytes(1000, 4) + request_bytes(2000, 4))
    assert select_batch(pend, 0, 10 ** 12, 1) == (1, request_bytes(1000, 4))


def test_head_that_does_not_fit_blocks_the_queue():
    pend = [_req(10 ** 6), _req(10)]
    small = request_bytes(10, 4)
    # the small request behind a large head waits: no overtaking
    assert select_batch(pend, 0, request_bytes(10 ** 6, 4) - 1, 8) == (0, 0)
    # memory in flight counts against the budget
    assert select_batch([_req(10)], 10 ** 9, 10 ** 9 + small - 1, 8) == (0, 0)
    assert select_batch([_req(10)], 10 ** 9, 10 ** 9 + small, 8) == (1, small)


def test_one_dtype_per_batch():
    pend = [_req(100), _req(100), _req(100, np.uint16), _req(100)]
    assert select_batch(pend, 0, 10 ** 12, 8)[0] == 2
    assert select_batch(pend[2:], 0, 10 ** 12, 8)[0] == 1


def test_request_bytes_grows_with_size_and_itemsize():
    assert request_bytes(100, 4) > request_bytes(100, 2)
    assert request_bytes(200, 4) == 2 * request_bytes(100, 4)


def test_idle_handles_stay_within_a_share_of_the_budget():
    assert keeps_buffers(100, 400, 4) and keeps_buffers(100, 400, 1)
    assert not keeps_buffers(101, 400, 4)
    assert keeps_buffers(400, 400, 1) and not keeps_buffers(401, 400, 1)
    assert keeps_buffers(0, 0, 0)


def test_batch_bounded_by_vertices_after_the_first():
    pend = [_req(3000), _req(3000), _req(3000), _req(100)]
    # the first request is always taken, even above the bound
    assert select_batch(pend, 0, 10 ** 12, 8, max_vertices=1000)[0] == 1
    assert select_batch(pend, 0, 10 ** 12, 8, max_vertices=6000)[0] == 2
    assert select_batch(pend, 0, 10 ** 12, 8, max_vertices=9100)[0] == 4
    assert select_batch(pend, 0, 10 ** 12, 8, max_vertices=None)[0] == 4


def test_only_a_backlog_is_batched():
    pend = [_req(100)] * 6
    assert select_batch(pend, 0, 10 ** 12, 8, batch_above=4)[0] == 6
    assert select_batch(pend[:4], 0, 10 ** 12, 8, batch_above=4)[0] == 1
    assert select_batch(pend[:4], 0, 10 ** 12, 8)[0] == 4
    assert select_batch(pend[:5], 0, 10 ** 12, 8, batch_above=4)[0] == 5
