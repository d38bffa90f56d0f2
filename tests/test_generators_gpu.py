"""Row f4, persistent 1-cycle generators (Sec. 8) through the C ABI.

A grid made with ``generators=True`` returns, for every D1 pair (tau,
sigma_j), a set of edges.  The generator is not unique: the paper's
propagation (Alg. 3) stops on one cycle, the GPU's reduction, which expands
every regular edge of a column, on another.  So the GPU is graded on the
three properties that define a generator, as the oracle's own generators are
in tests/test_oracle_sandwich.py:

- the edges form a 1-cycle (every vertex has even degree);
- its highest edge in the lexicographic order is the birth edge tau;
- adding the boundary of sigma_j gives a sum (mod 2) of boundaries of
  triangles that come before sigma_j.

The pairs themselves must equal the oracle's, simplex for simplex.
"""
import numpy as np
import pytest

import oracle
import synthfields as sf
from tests import bruteforce as bf
from tests.gpu_helpers import compare
from tests.test_oracle_sandwich import _Complex

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dms():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2206_13932_gb300 as m
    m.build()
    return m


def _gpu(dms, v, virtual_max=True):
    import torch
    nz, ny, nx = v.shape
    with dms.Grid((nx, ny, nz), v.dtype, virtual_max=virtual_max, generators=True) as g:
        g.compute(torch.from_numpy(np.ascontiguousarray(v)).cuda())
        return {d: g.fetch(d) for d in range(3)}, g.generators()


def _check(v, diag, gens, rows):
    compare(v, diag, rows)
    d1 = {(int(r[1]), int(r[2])) for r in rows if r[0] == 1 and not r[5]}
    assert set(gens) == d1
    cx = _Complex(v)
    edges = sorted((s for s in cx.by_id.values() if len(s) == 2), key=cx.lex)
    eidx = {s: i for i, s in enumerate(edges)}
    tris = sorted((s for s in cx.by_id.values() if len(s) == 3), key=cx.lex)

    def bvec(t):
        return sum(1 << eidx[t - {u}] for u in t)

    basis, ti = bf.GF2Basis(), 0
    for birth, death in sorted(gens, key=lambda p: cx.lex(cx.by_id[(2, p[1])])):
        t = cx.by_id[(2, death)]
        while ti < len(tris) and cx.lex(tris[ti]) < cx.lex(t):   # triangles before sigma_j
            basis.add(bvec(tris[ti]))
            ti += 1
        cyc = [cx.by_id[(1, int(e))] for e in gens[(birth, death)]]
        assert len(set(cyc)) == len(cyc) > 0
        deg = {}
        for e in cyc:
            for u in e:
                deg[u] = deg.get(u, 0) ^ 1
        assert not any(deg.values()), "not a 1-cycle"
        assert max(cyc, key=cx.lex) == cx.by_id[(1, birth)], "highest edge is not the birth"
        vec = sum(1 << eidx[e] for e in cyc) ^ bvec(t)
        while vec and (vec.bit_length() - 1) in basis.piv:
            vec ^= basis.piv[vec.bit_length() - 1]
        assert vec == 0, "not homologous to the boundary of the death triangle"
    return len(gens)


def _rand(rng, shape, kind, dtype):
    nx, ny, nz = shape
    if kind == "perm":
        return rng.permutation(nx * ny * nz).astype(dtype).reshape(nz, ny, nx)
    if kind == "ties":
        return rng.integers(0, 4, (nz, ny, nx)).astype(dtype)
    return rng.random((nz, ny, nx)).astype(dtype)


@pytest.mark.parametrize("seed", range(3))
def test_random_tiny_grids(dms, seed):
    rng = np.random.default_rng(3300 + seed)
    checked = 0
    for t in range(15):
        shape = tuple(int(s) for s in rng.integers(2, 7, 3))
        kind = ["perm", "ties", "float"][t % 3]
        dtype = [np.float32, np.uint16, np.float64][(t // 3) % 3]
        v = _rand(rng, shape, kind, dtype)
        vmax = t % 4 != 3
        diag, gens = _gpu(dms, v, vmax)
        rows, _ = oracle.sandwich(v, virtual_max=vmax)
        checked += _check(v, diag, gens, rows)
    assert checked > 20


@pytest.mark.parametrize("name", ["noise10", "mixture12", "recipe12_u16"])
def test_small_fields(dms, name):
    if name == "noise10":
        v = sf.white_noise((10, 10, 10), 31)
    elif name == "mixture12":
        v = sf.gaussian_mixture((12, 12, 12), 6, 32, noise=1e-3)
    else:
        v = sf.config_field("mixture512_u16", shape_xyz=(12, 12, 12))
    diag, gens = _gpu(dms, v)
    assert _check(v, diag, gens, oracle.pairsimplices(v)) > 0


def test_without_generators_the_call_is_refused(dms):
    import torch
    v = sf.white_noise((6, 5, 4), 33)
    with dms.Grid((6, 5, 4), v.dtype) as g:
        g.compute(torch.from_numpy(v).cuda())
        with pytest.raises(dms.DmsError) as e:
            g.generators()
        assert e.value.status == 6
