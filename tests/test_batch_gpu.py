"""Batches: many fields of their own shapes computed in one pass of the
pipeline (the disjoint union of the grids).  Each field's pairs must equal,
byte for byte, those of a single-grid compute of that field (the pairing is
exact integer work), and the oracle's on small fields."""
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


def _single(dms, v, mode=0):
    nz, ny, nx = v.shape
    with dms.Grid((nx, ny, nz), v.dtype, d1_mode=mode) as g:
        g.compute(v)
        return {d: g.fetch(d) for d in range(3)}


def _batch(dms, fields, mode=0, device=False):
    import torch
    shapes = [(f.shape[2], f.shape[1], f.shape[0]) for f in fields]
    with dms.Batch(shapes, fields[0].dtype, d1_mode=mode) as b:
        if device:
            b.compute([torch.from_numpy(f.copy()).cuda() for f in fields])
        else:
            b.compute(fields)
        res = b.results()
        st = b.stats()
    return res, st


def _same(a, b):
    for d in range(3):
        assert a[d].tobytes() == b[d].tobytes(), d


@pytest.mark.parametrize("dtype", [np.float32, np.uint16, np.float64])
def test_tiny_fields_match_single_and_oracle(dms, dtype):
    rng = np.random.default_rng(77)
    fields = []
    for t in range(24):
        shape = tuple(int(s) for s in rng.integers(1, 7, 3))
        if t % 3 == 0:
            v = rng.integers(0, 4, shape).astype(dtype)                      # ties
        elif t % 3 == 1:
            v = rng.permutation(int(np.prod(shape))).astype(dtype).reshape(shape)
        else:
            v = (rng.random(shape) * 1000).astype(dtype)
        fields.append(v)
    res, _ = _batch(dms, fields)
    for f, r in zip(fields, res):
        _same(r, _single(dms, f))
        compare(f, r, oracle.pairsimplices(f))


@pytest.mark.parametrize("mode", [0, 1, 3])
def test_serving_shapes_every_mode(dms, mode):
    fields = sf.serving_fields(20, seed0=5000, lo=8, hi=48)
    fields += [sf.white_noise(sh, 300 + i) for i, sh in enumerate(sf.serving_shapes(6, 301, 8, 40))]
    res, st = _batch(dms, fields, mode=mode, device=True)
    for f, r in zip(fields, res):
        _same(r, _single(dms, f, mode))


def test_one_field_batch_and_degenerate_fields(dms):
    v = sf.gaussian_mixture((33, 17, 21), 8, 3, noise=1e-3)
    res, _ = _batch(dms, [v])
    _same(res[0], _single(dms, v))
    fields = [np.zeros((1, 1, 1), np.float32), np.arange(5, dtype=np.float32).reshape(1, 1, 5),
              sf.white_noise((4, 3, 1), 9), np.full((2, 3, 4), 7.0, np.float32),
              sf.white_noise((9, 8, 7), 10)]
    res, _ = _batch(dms, fields)
    for f, r in zip(fields, res):
        _same(r, _single(dms, f))
        assert r[0]["essential"].sum() == 1      # one component per field


def test_offsets_and_refusals(dms):
    fields = [sf.white_noise((6, 5, 4), 1), sf.white_noise((3, 8, 2), 2)]
    shapes = [(6, 5, 4), (3, 8, 2)]
    with dms.Batch(shapes, np.float32) as b:
        b.compute(fields)
        pairs, ess = b.counts()
        for d in range(3):
            off = b.offsets(d)
            assert off[0] == 0 and off[-1] == pairs[d] + ess[d]
            assert np.all(np.diff(off) >= 0)
        with pytest.raises(dms.DmsError):
            b.reshape((4, 4, 4))
        # re-targeted to another batch: the same results as a fresh handle
        other = [sf.white_noise((7, 3, 9), 4), sf.white_noise((2, 2, 2), 5),
                 sf.white_noise((11, 6, 5), 6)]
        b.reshape([(f.shape[2], f.shape[1], f.shape[0]) for f in other]).compute(other)
        for f, r in zip(other, b.results()):
            _same(r, _single(dms, f))
    with dms.Grid((4, 4, 4), np.float32) as g:
        g.compute(sf.white_noise((4, 4, 4), 3))
        import ctypes
        off = (ctypes.c_int64 * 2)()
        assert g._lib.dms_batch_offsets(g._h, 0, off) == 6   # DMS_ERR_STATE


def test_batch_backward_matches_single(dms):
    import torch
    from paper_2206_13932_gb300.autograd import persistence_diagram, persistence_loss
    fields = [sf.gaussian_mixture(sh, 6, 40 + i, noise=1e-3)
              for i, sh in enumerate([(20, 16, 12), (9, 14, 11), (16, 16, 16)])]
    shapes = [(f.shape[2], f.shape[1], f.shape[0]) for f in fields]
    packed = torch.from_numpy(np.concatenate([f.reshape(-1) for f in fields])).cuda()
    packed.requires_grad_(True)
    b = dms.Batch(shapes, np.float32)
    loss = persistence_loss(persistence_diagram(packed, b), threshold=0.01)
    loss.backward()
    want = []
    for f in fields:
        t = torch.from_numpy(f.copy()).cuda().requires_grad_(True)
        g = dms.Grid((f.shape[2], f.shape[1], f.shape[0]), np.float32)
        persistence_loss(persistence_diagram(t, g), threshold=0.01).backward()
        want.append(t.grad.reshape(-1))
        g.close()
    # FP64 atomics may add a vertex's few terms in another order: equal up to rounding
    assert torch.allclose(packed.grad, torch.cat(want), rtol=1e-6, atol=1e-9)
    assert int((packed.grad != 0).sum()) > 0
    b.close()
