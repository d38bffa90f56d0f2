"""Bit-exact parity against the standard reduction itself (the oracle's fast
mode, ``oracle.fastpairs``, pinned equal to the textbook reduction) at sizes
the textbook mode cannot reach: every pair of D0, D1 and D2 by simplex id,
maximum vertices and raw value bits.

- 128^3 white noise (float32) and the 512^3 uint16 recipe at 128^3: the GPU
  in every D1 mode;
- the batching-and-serving workload: 64 of its 1024 fields (the 32 smallest
  and 32 drawn at random), computed one by one and as one batch;
- the differentiation workload: field 0 of the 8 x 128^3 batch, the pairing
  the backward pass uses.

The full-size configurations are checked against stored digests of the
same oracle's output in tests/test_zz_fullsize_gpu.py.

The oracle runs in a process pool (spawn) on the host's cores while the GPU
computes."""
import multiprocessing
import os

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
    oracle.build()
    return m


@pytest.fixture(scope="module")
def pool():
    ctx = multiprocessing.get_context("spawn")
    with ctx.Pool(max(1, min(16, (os.cpu_count() or 2) - 1))) as p:
        yield p


def _gpu(dms, values, mode=0):
    import torch
    nz, ny, nx = values.shape
    with dms.Grid((nx, ny, nz), values.dtype, d1_mode=mode) as g:
        g.compute(torch.from_numpy(np.ascontiguousarray(values)).cuda())
        return {d: g.fetch(d) for d in range(3)}


@pytest.mark.parametrize("name", ["noise128_f32", "recipe128_u16"])
def test_128_fields_against_the_standard_reduction(dms, pool, name):
    if name == "noise128_f32":
        v = sf.white_noise((128, 128, 128), 2)
    else:
        v = sf.config_field("mixture512_u16", shape_xyz=(128, 128, 128))
    job = pool.apply_async(oracle.fastpairs, (v,))
    diags = {mode: _gpu(dms, v, mode) for mode in (0, 1, 2, 3)}
    rows = job.get()
    assert sum(1 for r in rows if r[0] == 1) > 100000
    for mode, diag in diags.items():
        compare(v, diag, rows)


def test_serving_fields_against_the_standard_reduction(dms, pool):
    shapes = sf.serving_shapes(1024)
    size = np.array([a * b * c for a, b, c in shapes])
    order = np.argsort(size, kind="stable")
    rest = np.random.default_rng(4242).choice(order[32:], 32, replace=False)
    picks = sorted(set(order[:32].tolist()) | set(rest.tolist()))
    fields = [sf.serving_field(i) for i in picks]
    jobs = [pool.apply_async(oracle.fastpairs, (f,)) for f in fields]
    alone = [_gpu(dms, f) for f in fields]
    with dms.Batch([(f.shape[2], f.shape[1], f.shape[0]) for f in fields], np.float32) as b:
        b.compute(fields)
        batched = b.results()
    for f, a, bt, job in zip(fields, alone, batched, jobs):
        rows = job.get()
        compare(f, a, rows)
        compare(f, bt, rows)


def test_differentiation_pairing_against_the_standard_reduction(dms, pool):
    import torch
    from paper_2206_13932_gb300 import autograd
    v = sf.gaussian_mixture((128, 128, 128), 16, 5000, noise=0.0, dtype=np.float32)
    job = pool.apply_async(oracle.fastpairs, (v,))
    t = torch.from_numpy(v).cuda().requires_grad_(True)
    dg = autograd.persistence_diagram(t)
    loss = autograd.persistence_loss(dg, 0.01)
    loss.backward()
    got = set()
    for d in range(3):
        for b, e, ess in zip(dg[d].birth_simplex.cpu().numpy(), dg[d].death_simplex.cpu().numpy(),
                             dg[d].essential.cpu().numpy()):
            got.add((d, int(b), int(e), int(ess)))
    want = {(int(r[0]), int(r[1]), int(r[2]), int(r[5])) for r in job.get()}
    assert got == want
    # the gradient lands only on the maximum vertices of the pairs in the loss
    g = t.grad.reshape(-1).cpu().numpy()
    support = set()
    for d in (0, 2):
        p = (dg[d].death - dg[d].birth).detach().cpu().numpy()
        keep = (~dg[d].essential.cpu().numpy()) & (p > 0.01)
        support |= set(dg[d].birth_vertex.cpu().numpy()[keep].tolist())
        support |= set(dg[d].death_vertex.cpu().numpy()[keep].tolist())
    assert set(np.nonzero(g)[0].tolist()) <= support
