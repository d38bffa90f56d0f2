"""Parity of the CUDA path (through the C ABI) with the oracle.

The bar is bit-exact: every pair's birth/death simplex ids, maximum vertices,
raw value bits and the infinite classes equal the oracle's standard
reduction of the lexicographic filtration (integer pairing work, no
tolerance)."""
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


def _gpu(dms, values, on_device=True):
    import torch
    nz, ny, nx = values.shape
    t = torch.from_numpy(values.copy())
    if on_device:
        t = t.cuda()
    with dms.Grid((nx, ny, nz), values.dtype) as g:
        g.compute(t)
        return {d: g.fetch(d) for d in range(3)}, g.stats()


def _rand(rng, shape_xyz, kind, dtype=np.float32):
    nx, ny, nz = shape_xyz
    n = nx * ny * nz
    if kind == "perm":
        return rng.permutation(n).astype(dtype).reshape(nz, ny, nx)
    if kind == "ties":
        return rng.integers(0, 4, (nz, ny, nx)).astype(dtype)
    return rng.random((nz, ny, nx)).astype(dtype)


@pytest.mark.parametrize("seed", range(4))
def test_random_tiny_grids(dms, seed):
    rng = np.random.default_rng(1000 + seed)
    for t in range(40):
        shape = tuple(int(s) for s in rng.integers(1, 7, 3))
        kind = ["perm", "ties", "float"][t % 3]
        dtype = [np.float32, np.uint16, np.float64][(t // 3) % 3]
        v = _rand(rng, shape, kind, dtype)
        diag, _ = _gpu(dms, v)
        compare(v, diag, oracle.pairsimplices(v))


def test_mixture32_f32(dms):
    """32^3 float32: 16 Gaussians + 1e-3 noise, seed 1 (the smooth workload)."""
    v = sf.config_field("mixture32_f32")
    diag, st = _gpu(dms, v)
    compare(v, diag, oracle.pairsimplices(v))


@pytest.mark.parametrize("shape", [(40, 36, 33), (29, 47, 31)])
def test_white_noise_ragged(dms, shape):
    """White noise spanning several 2048-vertex tiles with a ragged tail."""
    v = sf.white_noise(shape, 21)
    diag, st = _gpu(dms, v)
    compare(v, diag, oracle.pairsimplices(v))


def test_quantized_u16_heavy_ties(dms):
    g = sf.gaussian_mixture((44, 38, 35), 12, 5, noise=0.05, noise_rel=True, dtype=None)
    v = (sf.quantize_u16(g) // 512).astype(np.uint16)   # ~128 levels: heavy ties
    diag, _ = _gpu(dms, v)
    compare(v, diag, oracle.pairsimplices(v))


def test_float64_mixture(dms):
    v = sf.gaussian_mixture((30, 26, 28), 10, 9, noise=1e-4, dtype=np.float64)
    diag, _ = _gpu(dms, v)
    compare(v, diag, oracle.pairsimplices(v))


def test_host_input_path(dms):
    v = sf.white_noise((20, 17, 15), 4)
    diag, _ = _gpu(dms, v, on_device=False)
    compare(v, diag, oracle.pairsimplices(v))


@pytest.mark.parametrize("shape", [(1, 1, 1), (5, 1, 1), (1, 7, 1), (1, 1, 6), (9, 8, 1),
                                   (1, 6, 7), (2, 2, 2), (64, 2, 2)])
def test_degenerate_shapes(dms, shape):
    rng = np.random.default_rng(7)
    for kind in ("perm", "ties"):
        v = _rand(rng, shape, kind)
        diag, _ = _gpu(dms, v)
        compare(v, diag, oracle.pairsimplices(v))


def test_elevation_and_constant(dms):
    for v in (sf.ramp((17, 13, 11)), sf.constant((12, 9, 10))):
        diag, _ = _gpu(dms, v)
        assert len(diag[1]) == 0 and len(diag[2]) == 0
        assert len(diag[0]) == 1 and diag[0][0]["essential"] == 1 and diag[0][0]["birth_simplex"] == 0


def test_nan_is_rejected(dms):
    v = sf.white_noise((8, 8, 8), 3)
    v[3, 4, 5] = np.nan
    with pytest.raises(dms.DmsError) as e:
        _gpu(dms, v)
    assert e.value.status == 2


def test_signed_zero(dms):
    a = sf.white_noise((12, 11, 10), 5)
    a[a < 0.4] = 0.0
    b = a.copy()
    b[a == 0.0] = -0.0
    da, _ = _gpu(dms, a)
    db, _ = _gpu(dms, b)
    for d in range(3):
        assert np.array_equal(da[d][["birth_simplex", "death_simplex"]],
                              db[d][["birth_simplex", "death_simplex"]])


def test_iteration_limit_is_an_error(dms):
    """A descent longer than max_iters ends with DMS_ERR_ITER_LIMIT, no hang."""
    import torch
    v = sf.ramp((30, 30, 30))
    v[-1, -1, -1] = -1.0
    v[5, 5, 5] = -2.0         # two minima: long descending paths
    t = torch.from_numpy(v).cuda()
    with dms.Grid((30, 30, 30), np.float32, max_iters=2) as g:
        with pytest.raises(dms.DmsError) as e:
            g.compute(t)
        assert e.value.status == 5


def test_deterministic_and_reusable(dms):
    import torch
    v = sf.white_noise((24, 25, 26), 8)
    t = torch.from_numpy(v).cuda()
    with dms.Grid((24, 25, 26), np.float32) as g:
        outs = []
        for _ in range(3):
            g.compute(t)
            outs.append([g.fetch(d).tobytes() for d in range(3)])
    assert outs[0] == outs[1] == outs[2]


def test_device_bytes_hold_the_grid_state_and_only_grow(dms):
    v = sf.white_noise((20, 18, 16), 4)
    with dms.Grid((20, 18, 16), np.float32) as g:
        before = g.device_bytes()
        g.compute(v)
        after = g.device_bytes()
        assert after >= before and after >= v.size * (1 + 4 + 48)   # flags, ranks, records
        w = sf.white_noise((40, 30, 20), 5)
        g.reshape((40, 30, 20)).compute(w)
        assert g.device_bytes() > after
