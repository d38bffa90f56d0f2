"""At the benchmark's full sizes, independent routes through the D1
reduction agree byte for byte: the default (rounds, then the asynchronous
tail), rounds only, and the anti-transposed (cohomology) reduction; with
the tunables at the other candidates as well.  The pairing is unique, so any
scheduling or ownership race would show as a difference here."""
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


def _run(dms, t, shape, dtype, mode=0, tuning=None):
    from paper_2206_13932_gb300 import autotune as at
    with dms.Grid(shape, dtype, d1_mode=mode) as g:
        if tuning:
            vals = list(at.DEFAULT)
            for k, v in tuning.items():
                vals[at.TUNABLES.index(k)] = v
            at.set_tuning(g, vals)
        g.compute(t)
        return [g.fetch(d).tobytes() for d in range(3)], g.stats()


@pytest.mark.parametrize("name", ["noise256", "mixture_u16_256"])
def test_reduction_routes_agree(dms, name):
    import torch
    if name == "noise256":
        v = sf.white_noise((256, 256, 256), 2)
    else:
        v = sf.config_field("mixture512_u16", shape_xyz=(256, 256, 256), device="cuda")
    t = torch.from_numpy(np.ascontiguousarray(v)).cuda()
    shape = (256, 256, 256)
    want, st = _run(dms, t, shape, v.dtype)
    assert st["d1_columns"] > 10 ** 6
    routes = [dict(mode=0, tuning={"red_async": 0}),
              dict(mode=0, tuning={"red_block_below": 8192}),
              dict(mode=0, tuning={"pls_sort": 0, "trace_heap": 32}),
              dict(mode=2)]
    for r in routes:
        got, _ = _run(dms, t, shape, v.dtype, **r)
        for d in range(3):
            assert got[d] == want[d], (name, r, d)
