"""Pins of the fast-mode standard reduction (``oracle.fastpairs``).

Fast mode must give exactly the pairs of the textbook standard reduction
(``oracle.pairsimplices``), zero-persistence pairs and infinite classes
included: clearing, apparent columns kept implicit and the streamed
filtration change how the reduction is carried out, not its pivots
(Sec. 2.5; Sec. 4, observation (a)).  Checked against the textbook mode on
every vertex order of the 2x2x2 grid and on random, tied, degenerate and
mixed-dtype grids up to 16^3; against the pairing-uniqueness rank formula
directly on the smallest grids; and at 32^3 against the union-find special
cases and the Euler characteristic of every sub-level set.
"""
import itertools
import zlib

import numpy as np
import pytest

import oracle
import synthfields as sf
from tests import bruteforce as bf


def _rand(rng, shape, kind):
    nx, ny, nz = shape
    n = nx * ny * nz
    if kind == "perm":
        return (rng.permutation(n) - n // 2).astype(np.float32).reshape(nz, ny, nx)
    if kind == "ties":
        return rng.integers(0, 3, (nz, ny, nx)).astype(np.uint16)
    if kind == "f64":
        return rng.standard_normal((nz, ny, nx))
    return (rng.random((nz, ny, nx)) - 0.5).astype(np.float32)


def _rows(rows):
    return {(int(r[0]), int(r[1]), int(r[2]), int(r[3]), int(r[4]), int(r[5])) for r in rows}


def _same(v, keep_zero):
    a = _rows(oracle.pairsimplices(v, keep_zero=keep_zero))
    b = oracle.fastpairs(v, keep_zero=keep_zero)
    assert len(_rows(b)) == len(b), "duplicate rows"
    assert _rows(b) == a


def test_every_order_of_a_cube():
    """All 8! vertex orders of the 2x2x2 grid, zero-persistence pairs kept."""
    for perm in itertools.permutations(range(8)):
        _same(np.array(perm, dtype=np.float32).reshape(2, 2, 2), True)


@pytest.mark.parametrize("shape,kind,trials", [
    ((2, 2, 2), "ties", 30), ((3, 2, 2), "perm", 20), ((3, 3, 3), "float", 15),
    ((4, 3, 3), "ties", 10), ((5, 4, 3), "perm", 8), ((6, 5, 4), "f64", 6),
    ((1, 1, 1), "float", 2), ((9, 1, 1), "perm", 3), ((1, 7, 1), "ties", 3),
    ((1, 1, 8), "float", 3), ((6, 5, 1), "perm", 4), ((1, 5, 6), "ties", 4),
    ((5, 1, 6), "f64", 4)])
@pytest.mark.parametrize("keep_zero", [False, True])
def test_equals_textbook_on_random_grids(shape, kind, trials, keep_zero):
    rng = np.random.default_rng(zlib.crc32(repr((shape, kind, keep_zero)).encode()))
    for _ in range(trials):
        _same(_rand(rng, shape, kind), keep_zero)


@pytest.mark.parametrize("name", ["noise16", "mixture16", "u16_16", "constant", "ramp"])
def test_equals_textbook_on_recipes(name):
    if name == "noise16":
        v = sf.white_noise((16, 15, 14), 21)
    elif name == "mixture16":
        v = sf.gaussian_mixture((16, 16, 16), 6, 22, noise=1e-3)
    elif name == "u16_16":
        v = sf.quantize_u16(sf.gaussian_mixture((16, 16, 16), 8, 23, noise=0.05, dtype=None,
                                                noise_rel=True)) // 256
    elif name == "constant":
        v = sf.constant((7, 6, 5))
    else:
        v = sf.ramp((7, 6, 5))
    _same(v, False)


def test_equals_rank_formula():
    """Independent of the textbook mode: every pair by simplex id, zero
    persistence included, equals the pairing-uniqueness rank formula."""
    rng = np.random.default_rng(31)
    for shape, kind, trials in [((2, 2, 2), "perm", 12), ((3, 2, 2), "ties", 6),
                                ((2, 3, 2), "float", 6)]:
        for _ in range(trials):
            v = _rand(rng, shape, kind)
            order = bf.lex_order(bf.freudenthal_simplices(shape), bf.vertex_keys(v))
            want, paired = set(), set()
            for i, j in bf.pairing_by_ranks(order):
                want.add((len(order[i]) - 1, bf.simplex_id(shape, order[i]),
                          bf.simplex_id(shape, order[j])))
                paired |= {i, j}
            rows = oracle.fastpairs(v, keep_zero=True)
            assert {(int(r[0]), int(r[1]), int(r[2])) for r in rows if not r[5]} == want
            assert {(int(r[0]), int(r[1])) for r in rows if r[5]} == \
                {(len(order[i]) - 1, bf.simplex_id(shape, order[i]))
                 for i in range(len(order)) if i not in paired}


def test_union_find_cases_and_euler_characteristic_at_32():
    """32^3 noise: D0 and D2 equal the union-find special cases, exactly one
    infinite class (the global minimum), and at every vertex rank the counts
    of classes alive give the Euler characteristic of the sub-level set."""
    v = sf.white_noise((32, 32, 32), 24)
    rows = oracle.fastpairs(v)
    fin = {(int(r[0]), int(r[1]), int(r[2])) for r in rows if not r[5]}
    assert {(int(r[0]), int(r[1]), int(r[2])) for r in oracle.kruskal_d0(v) if not r[5]} == \
        {p for p in fin if p[0] == 0}
    assert {(int(r[0]), int(r[1]), int(r[2])) for r in oracle.kruskal_d2(v)} == \
        {p for p in fin if p[0] == 2}
    ess = [r for r in rows if r[5]]
    assert len(ess) == 1 and int(ess[0][0]) == 0 and int(ess[0][1]) == int(np.argmin(v))
    # chi(sub-level set at vertex rank t) = sum_d (-1)^d (#classes of dim d alive at t)
    flat = v.reshape(-1)
    rank = np.empty(flat.size, np.int64)
    rank[np.lexsort((np.arange(flat.size), flat))] = np.arange(flat.size)
    alive = np.zeros(flat.size + 1, np.int64)
    for r in rows:
        s = (-1) ** int(r[0])
        alive[rank[r[3]]] += s
        if not r[5]:
            alive[rank[r[4]]] -= s
    chi_pairs = np.cumsum(alive)[:-1]
    # chi of the sub-level set from the simplex counts of the lower stars
    nz, ny, nx = v.shape
    counts = np.zeros(flat.size, np.int64)
    for dim, mult in enumerate((1, 7, 12, 6)):
        for sid in range(flat.size * mult):
            vs = oracle.simplex_vertices((nx, ny, nz), dim, sid) if dim else (sid,)
            if vs is None:
                continue
            counts[max(rank[list(vs)])] += (-1) ** dim
    assert np.array_equal(chi_pairs, np.cumsum(counts))
