"""Row f4, the option without the virtual maximum (Sec. 5.2 "Domains with
boundary", App. A), through the C ABI against the oracle that runs the
method's own steps with the same option (``oracle.sandwich(values,
virtual_max=False)``; its parity is partly pinned, see
tests/test_oracle_sandwich.py): every pair by simplex id, maximum vertices
and raw value bits, the infinite classes of dimension 2 (2-saddles whose
column reduces to zero) and of dimension 3 (maxima left unpaired, listed at
the end of the D2 list), in every D1 mode, single grids and batches."""
import numpy as np
import pytest

import oracle
import synthfields as sf
from tests.gpu_helpers import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dms():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2206_13932_gb300 as m
    m.build()
    return m


def _gpu(dms, values, mode=0):
    import torch
    nz, ny, nx = values.shape
    with dms.Grid((nx, ny, nz), values.dtype, d1_mode=mode, virtual_max=False) as g:
        g.compute(torch.from_numpy(np.ascontiguousarray(values)).cuda())
        diag = {d: g.fetch(d) for d in range(3)}
        counts = g.counts()
    return diag, counts


def _rand(rng, shape, kind, dtype):
    nx, ny, nz = shape
    n = nx * ny * nz
    if kind == "perm":
        return rng.permutation(n).astype(dtype).reshape(nz, ny, nx)
    if kind == "ties":
        return rng.integers(0, 4, (nz, ny, nx)).astype(dtype)
    return rng.random((nz, ny, nx)).astype(dtype)


@pytest.mark.parametrize("seed", range(3))
def test_random_tiny_grids(dms, seed):
    rng = np.random.default_rng(2200 + seed)
    infinite3 = 0
    for t in range(36):
        shape = tuple(int(s) for s in rng.integers(1, 8, 3))
        kind = ["perm", "ties", "float"][t % 3]
        dtype = [np.float32, np.uint16, np.float64][(t // 3) % 3]
        v = _rand(rng, shape, kind, dtype)
        rows, _ = oracle.sandwich(v, virtual_max=False)
        for mode in (1, 2, 3):
            diag, counts = _gpu(dms, v, mode)
            compare(v, diag, rows)
            assert counts[1][3] == sum(1 for r in rows if r[5] and r[0] == 3)
        infinite3 += sum(1 for r in rows if r[5] and r[0] == 3)
    assert infinite3 > 0        # the cases hold maxima left unpaired


@pytest.mark.parametrize("name", ["noise24_f32", "mixture32_f32", "recipe32_u16"])
def test_medium_fields(dms, name):
    if name == "noise24_f32":
        v = sf.white_noise((24, 23, 22), 71)
    elif name == "mixture32_f32":
        v = sf.config_field("mixture32_f32")
    else:
        v = sf.config_field("mixture512_u16", shape_xyz=(32, 32, 32))
    rows, _ = oracle.sandwich(v, virtual_max=False)
    assert any(r[5] and r[0] == 2 for r in rows) or name != "noise24_f32"
    for mode in (0, 1, 2, 3):
        diag, _ = _gpu(dms, v, mode)
        compare(v, diag, rows)


def test_batch_equals_single_grids(dms):
    fields = [sf.white_noise(sh, 80 + i) for i, sh in
              enumerate([(9, 7, 5), (12, 3, 10), (1, 6, 6), (16, 16, 4)])]
    fields.append(sf.gaussian_mixture((20, 18, 16), 6, 85, noise=1e-3))
    with dms.Batch([(f.shape[2], f.shape[1], f.shape[0]) for f in fields], np.float32,
                   virtual_max=False) as b:
        b.compute(fields)
        got = b.results()
    for f, res in zip(fields, got):
        rows, _ = oracle.sandwich(f, virtual_max=False)
        compare(f, res, rows)
        alone, _ = _gpu(dms, f)
        for d in range(3):
            assert res[d].tobytes() == alone[d].tobytes()
