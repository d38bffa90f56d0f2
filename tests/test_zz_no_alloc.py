"""The allocation-free classification entry point, dms_classify_static.

Some callers cannot let a library allocate device memory (a process that
hands all of it to its own pool, a fixed memory budget, a latency-critical
pipeline where an allocation would stall other streams).  For them the C ABI
offers the classification step with its scratch in a fixed array inside the
library.  This test calls it through the C ABI, twice in a row, and checks it
against the existing entry point, dms_compute_diagram: the PL-critical
vertices it lists are exactly the maximum vertices of the simplices of the
diagram (every critical simplex is paired or essential, and only PL-critical
vertices carry critical simplices), and their number is the diagram's count
of critical vertices.  The comparison is exact (integer work).

This file is collected last so that a run stopping at the first failure has
run every other test before it; it also passes alone in a fresh process.
"""
import ctypes

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


def _existing(dms, v):
    """Critical vertex set and count from the full diagram entry point."""
    import torch
    nz, ny, nx = v.shape
    with dms.Grid((nx, ny, nz), v.dtype) as g:
        g.compute(torch.from_numpy(v).cuda())
        verts = set()
        for d in range(3):
            p = g.fetch(d)
            verts |= set(int(x) for x in p["birth_vertex"])
            verts |= set(int(x) for x in p["death_vertex"] if x >= 0)
        return verts, g.stats()["critical_vertices"]


def _static_call(dms, t, cap):
    """One call of dms_classify_static through the C ABI."""
    import torch
    lib = dms.load()
    nz, ny, nx = t.shape
    code = {torch.uint16: 0, torch.float32: 1, torch.float64: 2}[t.dtype]
    flags = torch.full((t.numel(),), 0xEE, dtype=torch.uint8, device="cuda")
    crit = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    n = ctypes.c_int64(-1)
    st = lib.dms_classify_static(ctypes.c_void_p(t.data_ptr()), code, nx, ny, nz,
                                 ctypes.c_void_p(flags.data_ptr()),
                                 ctypes.c_void_p(crit.data_ptr()), cap, ctypes.byref(n),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, n.value, flags.cpu().numpy(), crit.cpu().numpy()


@pytest.mark.parametrize("case", ["noise", "mixture_u16"])
def test_matches_existing_entry_point_twice(dms, case):
    import torch
    if case == "noise":
        v = sf.white_noise((45, 37, 33), 12)     # several 2048-vertex tiles, ragged tail
    else:
        g = sf.gaussian_mixture((40, 38, 31), 10, 4, noise=0.05, noise_rel=True, dtype=None)
        v = sf.quantize_u16(g)
    want, want_n = _existing(dms, v)
    t = torch.from_numpy(v).cuda()
    cap = v.size
    outs = []
    for _ in range(2):                           # the array keeps the last call's contents
        st, n, flags, crit = _static_call(dms, t, cap)
        assert st == 0, dms.STATUS.get(st, st)
        assert n == want_n == len(want)
        listed = crit[:n]
        assert np.all(np.diff(listed) > 0)       # increasing ids
        assert set(int(x) for x in listed) == want
        assert np.all(crit[n:] == -7)            # nothing written past the count
        flagged = np.nonzero(flags & 0x10)[0]
        assert np.array_equal(flagged, listed)
        assert np.all(flags & 0xE0 == 0)
        outs.append((n, flags.copy(), listed.copy()))
    assert outs[0][0] == outs[1][0]
    assert np.array_equal(outs[0][1], outs[1][1]) and np.array_equal(outs[0][2], outs[1][2])


def test_rejects_sizes_beyond_the_fixed_scratch(dms):
    import torch
    lib = dms.load()
    t = torch.zeros(8, dtype=torch.float32, device="cuda")
    n = ctypes.c_int64(0)
    st = lib.dms_classify_static(ctypes.c_void_p(t.data_ptr()), 1, 1 << 10, 1 << 10, 1 << 9,
                                 ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                 0, ctypes.byref(n), None)
    assert st == 1                               # DMS_ERR_INVALID_ARG, nothing launched


def test_capacity_too_small_is_reported(dms):
    import torch
    v = sf.white_noise((20, 18, 16), 5)
    t = torch.from_numpy(v).cuda()
    st, n, _, crit = _static_call(dms, t, 3)
    assert st == 7 and n > 3                     # DMS_ERR_CAPACITY, count still reported
    assert np.all(crit == -7)
