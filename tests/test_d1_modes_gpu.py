"""The three D1 reductions -- the traced columns (1), their anti-transpose
(2, persistent cohomology) and the lazy columns that are expanded only as far
as their pivots (3, Alg. 3's interleaving of propagation and reduction) --
give the oracle's pairs, and one another's bit for bit on larger fields."""
import os

import numpy as np
import pytest

import oracle
import synthfields as sf
from tests.gpu_helpers import compare

pytestmark = pytest.mark.gpu

MODES = (1, 2, 3)


@pytest.fixture(scope="module")
def dms():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2206_13932_gb300 as m
    m.build()
    return m


def _run(dms, v, mode):
    import torch
    nz, ny, nx = v.shape
    with dms.Grid((nx, ny, nz), v.dtype, d1_mode=mode) as g:
        g.compute(torch.from_numpy(v.copy()).cuda())
        return {d: g.fetch(d) for d in range(3)}, g.stats()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("seed", range(2))
def test_tiny_grids(dms, mode, seed):
    rng = np.random.default_rng(2000 + seed)
    for t in range(30):
        shape = tuple(int(s) for s in rng.integers(1, 8, 3))
        dtype = [np.float32, np.uint16, np.float64][t % 3]
        if t % 2:
            v = rng.integers(0, 5, shape[::-1]).astype(dtype)          # heavy ties
        else:
            v = rng.permutation(int(np.prod(shape))).astype(dtype).reshape(shape[::-1])
        diag, _ = _run(dms, v, mode)
        compare(v, diag, oracle.pairsimplices(v))


@pytest.mark.parametrize("mode", MODES)
def test_oracle_sized_fields(dms, mode):
    fields = [sf.config_field("mixture32_f32"),
              sf.white_noise((40, 36, 33), 5),
              sf.quantize_u16(sf.gaussian_mixture((30, 34, 29), 12, 8)) >> 10]   # 6-bit ties
    for v in fields:
        diag, _ = _run(dms, v, mode)
        compare(v, diag, oracle.pairsimplices(v))


@pytest.mark.parametrize("name,make", [
    ("noise96", lambda: sf.white_noise((96, 96, 96), 11)),
    ("mixture80", lambda: sf.gaussian_mixture((80, 80, 80), 16, 12)),
    ("mixture_u16_72", lambda: sf.config_field("mixture512_u16", shape_xyz=(72, 72, 72))),
])
def test_modes_agree(dms, name, make):
    v = make()
    if not isinstance(v, np.ndarray):
        v = v.cpu().numpy()
    res = {m: _run(dms, v, m) for m in MODES}
    for m in MODES[1:]:
        for d in range(3):
            assert res[m][0][d].tobytes() == res[1][0][d].tobytes(), (name, m, d)
    assert res[3][1]["d1_columns"] == res[1][1]["d1_columns"]


def test_lazy_pool_regrowth(dms):
    """A pool far too small for the columns: the lazy path compacts and
    regrows it between rounds, and the pairs do not change."""
    v = sf.white_noise((48, 40, 44), 21)
    want, _ = _run(dms, v, 1)
    os.environ["DMS_D1_POOL_ENTRIES"] = "4096"
    try:
        got, st = _run(dms, v, 3)
    finally:
        del os.environ["DMS_D1_POOL_ENTRIES"]
    assert st["d1_pool_grows"] > 0
    for d in range(3):
        assert got[d].tobytes() == want[d].tobytes()


def test_lazy_scratch_retries(dms):
    """Columns of a smooth field whose expansions outgrow the first scratch
    are advanced again with larger scratch; the pairs do not change."""
    v = sf.gaussian_mixture((64, 64, 64), 6, 31, noise=1e-4)
    want, _ = _run(dms, v, 1)
    got, st = _run(dms, v, 3)
    assert st["d1_trace_overflow"] > 0
    for d in range(3):
        assert got[d].tobytes() == want[d].tobytes()


@pytest.mark.parametrize("level", ["1", "2"])
def test_lazy_retry_levels(dms, level):
    """The retried columns taken by the larger block scratch (level 1) or by
    the serial walk in global memory (level 2) give the same pairs."""
    v = sf.gaussian_mixture((64, 64, 64), 6, 31, noise=1e-4)
    want, _ = _run(dms, v, 1)
    os.environ["DMS_D1_LAZY_LEVEL"] = level
    try:
        got, st = _run(dms, v, 3)
    finally:
        del os.environ["DMS_D1_LAZY_LEVEL"]
    assert st["d1_trace_overflow"] > 0
    for d in range(3):
        assert got[d].tobytes() == want[d].tobytes()

