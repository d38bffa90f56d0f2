"""Pins of the sandwich oracle (``oracle/sandwich.c``), the method's own steps.

Every check compares it with something other than itself:

- With the virtual maximum, the sandwich returns the standard reduction's
  diagrams (Sec. 4.1 (c), Sec. 5): compared with ``oracle.pairsimplices`` on
  random, tied and permutation fields, and with the brute-force rank formula
  on the smallest grids.
- Its discrete gradient (Alg. 2) against the definition of a gradient (facet
  pairs inside one lower star, each simplex in at most one pair, no closed
  v-path) and two properties the method relies on: the critical simplices
  are exactly those of non-zero persistence (Sec. 4.1 (c)), and the critical
  simplices of a lower star count the reduced homology of its lower link
  (Sec. 2.6: the expansions of Robins et al. put every critical i-simplex in
  the lower star of a PL critical point of index i).
- Generators (Sec. 8), by brute force over GF(2): each is a 1-cycle, its
  highest edge is the birth edge, and it differs from the boundary of the
  death triangle by a sum of boundaries of earlier triangles.
- Without the virtual maximum (App. A), parity partly pinned: D0 does not
  change; on a field whose boundary lies below its interior, no pair between
  interior simplices changes; the highest maximum becomes an infinite class;
  every critical simplex is paired or infinite exactly once.
"""
import itertools
import zlib

import numpy as np
import pytest

import oracle
import synthfields as sf
from tests import bruteforce as bf


def _rand_field(rng, shape_xyz, kind):
    nx, ny, nz = shape_xyz
    if kind == "perm":
        return rng.permutation(nx * ny * nz).astype(np.float32).reshape(nz, ny, nx)
    if kind == "ties":
        return rng.integers(0, 3, (nz, ny, nx)).astype(np.uint16)
    return rng.random((nz, ny, nx))


def _pairs(rows):
    return {(int(r[0]), int(r[1]), int(r[2]), int(r[5])) for r in rows}


class _Complex:
    """The grid's simplices from the brute-force chain definition, keyed."""

    def __init__(self, values):
        nz, ny, nx = values.shape
        self.shape = (nx, ny, nz)
        self.keys = bf.vertex_keys(values)
        self.by_id = {}
        for s in bf.freudenthal_simplices(self.shape):
            self.by_id[(len(s) - 1, bf.simplex_id(self.shape, s))] = s

    def lex(self, s):
        return tuple(sorted((self.keys[v] for v in s), reverse=True))

    def top(self, s):
        return max(s, key=lambda v: self.keys[v])


# ------------------------------- with the virtual maximum: the plain diagrams

@pytest.mark.parametrize("shape,kind,trials", [
    ((2, 2, 2), "perm", 40), ((3, 2, 2), "ties", 30), ((3, 3, 3), "float", 20),
    ((4, 3, 3), "perm", 15), ((5, 4, 3), "ties", 10), ((6, 5, 4), "float", 6),
    ((7, 1, 5), "float", 6), ((1, 1, 9), "perm", 4)])
def test_sandwich_equals_standard_reduction(shape, kind, trials):
    rng = np.random.default_rng(zlib.crc32(repr((shape, kind)).encode()))
    for _ in range(trials):
        v = _rand_field(rng, shape, kind)
        rows, _ = oracle.sandwich(v)
        assert _pairs(rows) == _pairs(oracle.pairsimplices(v))


@pytest.mark.parametrize("name", ["noise", "mixture", "u16"])
def test_sandwich_equals_standard_reduction_larger(name):
    if name == "noise":
        v = sf.white_noise((12, 11, 10), 7)
    elif name == "mixture":
        v = sf.gaussian_mixture((14, 13, 12), 5, 3, noise=1e-3)
    else:
        v = sf.quantize_u16(sf.gaussian_mixture((12, 12, 12), 4, 9)) // 512
    rows, gens = oracle.sandwich(v)
    assert _pairs(rows) == _pairs(oracle.pairsimplices(v))
    assert set(gens) == {(int(r[1]), int(r[2])) for r in rows if r[0] == 1 and not r[5]}


@pytest.mark.parametrize("name", ["noise40", "recipe48_u16"])
def test_sandwich_equals_standard_reduction_medium(name):
    """At the larger sizes where the GPU tests use the sandwich in place of the
    slower reduction, the two still agree pair for pair."""
    if name == "noise40":
        v = sf.white_noise((40, 40, 40), 13)
    else:
        v = sf.quantize_u16(sf.gaussian_mixture((48, 48, 48), 24, 14, noise=0.05, dtype=None,
                                                noise_rel=True))
    rows, _ = oracle.sandwich(v)
    assert _pairs(rows) == _pairs(oracle.pairsimplices(v))


def test_sandwich_equals_standard_reduction_on_every_order_of_a_cube():
    """All 8! vertex orders of the 2x2x2 grid: the two oracles agree on every
    one, and without the virtual maximum D0 stays and the infinite classes
    still add up to the Euler characteristic."""
    for perm in itertools.permutations(range(8)):
        v = np.array(perm, dtype=np.float32).reshape(2, 2, 2)
        rows, _ = oracle.sandwich(v)
        assert _pairs(rows) == _pairs(oracle.pairsimplices(v)), perm
        off, _ = oracle.sandwich(v, virtual_max=False)
        assert {p for p in _pairs(off) if p[0] == 0} == {p for p in _pairs(rows) if p[0] == 0}
        assert sum((-1) ** int(r[0]) for r in off if r[5]) == 1


def test_sandwich_equals_rank_formula():
    """On the smallest grids, against the pairing uniqueness lemma directly."""
    rng = np.random.default_rng(11)
    for shape in [(2, 2, 2), (3, 2, 2)]:
        for _ in range(8):
            v = _rand_field(rng, shape, "perm")
            cx = _Complex(v)
            order = bf.lex_order(list(cx.by_id.values()), cx.keys)
            want = set()
            for i, j in bf.pairing_by_ranks(order):
                if cx.top(order[i]) != cx.top(order[j]):
                    want.add((len(order[i]) - 1, bf.simplex_id(cx.shape, order[i]),
                              bf.simplex_id(cx.shape, order[j])))
            rows, _ = oracle.sandwich(v)
            got = {(int(r[0]), int(r[1]), int(r[2])) for r in rows if not r[5]}
            assert got == want


# ------------------------------------------------------ the discrete gradient

def _reduced_betti(lower_link):
    """Reduced Betti numbers (dims -1..2) of a complex given as frozensets,
    over GF(2), with the empty simplex as the (-1)-cell."""
    cells = [[frozenset()]] + [[s for s in lower_link if len(s) == k + 1] for k in range(3)]
    index = [{s: i for i, s in enumerate(c)} for c in cells]
    ranks = [0] * 5          # ranks[k+1] = rank of the boundary of k-cells
    for k in range(3):
        basis = bf.GF2Basis()
        for s in cells[k + 1]:
            vec = 0
            for u in s:
                vec |= 1 << index[k][s - {u}]
            basis.add(vec)
        ranks[k + 1] = basis.rank
    return [len(cells[k + 1]) - ranks[k + 1] - ranks[k + 2] for k in range(-1, 3)]


@pytest.mark.parametrize("shape,kind,seed", [
    ((3, 3, 3), "float", 1), ((4, 3, 3), "ties", 2), ((4, 4, 3), "perm", 3),
    ((5, 4, 4), "float", 4), ((3, 3, 3), "ties", 5)])
def test_gradient_is_a_discrete_gradient(shape, kind, seed):
    v = _rand_field(np.random.default_rng(seed), shape, kind)
    cx = _Complex(v)
    grad = oracle.gradient(v)
    partner = {}
    for d, sid, pd, pid in grad:
        partner[(int(d), int(sid))] = None if pd < 0 else (int(pd), int(pid))
    assert set(partner) == set(cx.by_id)
    # a matching of facet pairs, inside one lower star
    for a, b in partner.items():
        if b is None:
            continue
        assert partner[b] == a
        sa, sb = cx.by_id[a], cx.by_id[b]
        lo, hi = (sa, sb) if len(sa) < len(sb) else (sb, sa)
        assert len(hi) == len(lo) + 1 and lo < hi
        assert cx.top(lo) == cx.top(hi)
    # no closed v-path: arrows up along pairs, down to the other facets
    for p in range(3):
        nodes = [k for k in cx.by_id if k[0] in (p, p + 1)]
        out = {k: [] for k in nodes}
        for k in nodes:
            s = cx.by_id[k]
            if k[0] == p and partner[k] is not None and partner[k][0] == p + 1:
                out[k].append(partner[k])
            if k[0] == p + 1:
                for u in s:
                    f = (p, bf.simplex_id(cx.shape, s - {u}))
                    if partner[k] != f:
                        out[k].append(f)
        indeg = {k: 0 for k in nodes}
        for k in nodes:
            for t in out[k]:
                indeg[t] += 1
        stack = [k for k in nodes if indeg[k] == 0]
        seen = 0
        while stack:
            k = stack.pop()
            seen += 1
            for t in out[k]:
                indeg[t] -= 1
                if indeg[t] == 0:
                    stack.append(t)
        assert seen == len(nodes), f"closed v-path between dimensions {p} and {p + 1}"
    # critical simplices are exactly those of non-zero persistence (Sec. 4.1 (c))
    crit = {k for k, b in partner.items() if b is None}
    rows = oracle.pairsimplices(v)
    cross = {(int(r[0]), int(r[1])) for r in rows} | \
        {(int(r[0]) + 1, int(r[2])) for r in rows if not r[5]}
    assert crit == cross
    # per lower star: critical p-simplices = reduced Betti number p-1 of the lower link
    for w in range(len(cx.keys)):
        star = [s for s in cx.by_id.values() if w in s and cx.top(s) == w]
        link = [s - {w} for s in star if len(s) > 1]
        counts = [0] * 4
        for (d, sid), b in partner.items():
            if b is None and cx.top(cx.by_id[(d, sid)]) == w:
                counts[d] += 1
        assert counts == _reduced_betti(link), w


# ------------------------------------------------------- generators (Sec. 8)

def _reduce(basis, vec):
    while vec:
        h = vec.bit_length() - 1
        if h not in basis.piv:
            return vec
        vec ^= basis.piv[h]
    return 0


@pytest.mark.parametrize("shape,kind,seed", [
    ((3, 3, 3), "float", 21), ((4, 3, 3), "perm", 22), ((4, 4, 3), "ties", 23),
    ((5, 4, 3), "float", 24), ((4, 4, 4), "perm", 25)])
@pytest.mark.parametrize("virtual_max", [True, False])
def test_generators_are_homologous_cycles(shape, kind, seed, virtual_max):
    v = _rand_field(np.random.default_rng(seed), shape, kind)
    cx = _Complex(v)
    rows, gens = oracle.sandwich(v, virtual_max=virtual_max)
    assert set(gens) == {(int(r[1]), int(r[2])) for r in rows if r[0] == 1 and not r[5]}
    edges = sorted((s for s in cx.by_id.values() if len(s) == 2), key=cx.lex)
    eidx = {s: i for i, s in enumerate(edges)}
    tris = sorted((s for s in cx.by_id.values() if len(s) == 3), key=cx.lex)

    def bvec(t):
        return sum(1 << eidx[t - {u}] for u in t)

    for (birth, death), cycle in gens.items():
        cyc = [cx.by_id[(1, e)] for e in cycle]
        assert len(set(cyc)) == len(cyc) > 0
        deg = {}
        for e in cyc:
            for u in e:
                deg[u] = deg.get(u, 0) ^ 1
        assert not any(deg.values()), "not a 1-cycle"
        assert max(cyc, key=cx.lex) == cx.by_id[(1, birth)], "highest edge is not the birth"
        t = cx.by_id[(2, death)]
        basis = bf.GF2Basis()
        for u in tris:
            if cx.lex(u) >= cx.lex(t):
                break
            basis.add(bvec(u))
        vec = sum(1 << eidx[e] for e in cyc) ^ bvec(t)
        assert _reduce(basis, vec) == 0, "not homologous to the death triangle's boundary"


# ------------------------------------ without the virtual maximum (App. A)

def _low_boundary_field(rng, shape_xyz, kind):
    """Interior values in [2, 3), boundary values in [0, 1): every boundary
    vertex lies below every interior vertex."""
    nx, ny, nz = shape_xyz
    z, y, x = np.meshgrid(range(nz), range(ny), range(nx), indexing="ij")
    inner = (x > 0) & (x < nx - 1) & (y > 0) & (y < ny - 1) & (z > 0) & (z < nz - 1)
    if kind == "ties":
        v = rng.integers(0, 4, (nz, ny, nx)) + np.where(inner, 8, 0)
        return v.astype(np.uint16), inner.reshape(-1)
    return (rng.random((nz, ny, nx)) + np.where(inner, 2.0, 0.0)), inner.reshape(-1)


@pytest.mark.parametrize("shape,kind,seed", [
    ((5, 5, 5), "float", 31), ((6, 5, 4), "float", 32), ((6, 6, 5), "ties", 33),
    ((7, 5, 5), "float", 34), ((5, 5, 5), "ties", 35)])
def test_without_virtual_maximum_interior_pairs_unchanged(shape, kind, seed):
    v, inner = _low_boundary_field(np.random.default_rng(seed), shape, kind)
    on, gon = oracle.sandwich(v, virtual_max=True)
    off, goff = oracle.sandwich(v, virtual_max=False)

    def interior(rows):
        return {(int(r[0]), int(r[1]), int(r[2])) for r in rows
                if not r[5] and inner[r[3]] and inner[r[4]]}
    a, b = interior(on), interior(off)
    assert a == b and len(a) > 0
    for d, bi, de in a:
        if d == 1:
            assert gon[(bi, de)] == goff[(bi, de)]


@pytest.mark.parametrize("shape,kind,seed", [
    ((4, 4, 4), "float", 41), ((5, 4, 3), "ties", 42), ((6, 5, 5), "perm", 43),
    ((3, 3, 3), "float", 44), ((6, 6, 6), "float", 45), ((2, 2, 2), "perm", 46)])
def test_without_virtual_maximum_invariants(shape, kind, seed):
    v = _rand_field(np.random.default_rng(seed), shape, kind)
    on, _ = oracle.sandwich(v, virtual_max=True)
    off, _ = oracle.sandwich(v, virtual_max=False)
    # D0 does not depend on the outer boundary
    assert {p for p in _pairs(on) if p[0] == 0} == {p for p in _pairs(off) if p[0] == 0}
    # with the virtual maximum, the global minimum is the only infinite class
    assert [int(r[0]) for r in on if r[5]] == [0]
    # every critical simplex is paired or infinite exactly once
    grad = oracle.gradient(v)
    crit = sorted((int(d), int(s)) for d, s, pd, _ in grad if pd < 0)
    seen = sorted([(int(r[0]), int(r[1])) for r in off] +
                  [(int(r[0]) + 1, int(r[2])) for r in off if not r[5]])
    assert seen == crit
    # the infinite classes still add up to the Euler characteristic of the cube
    ess = [int(r[0]) for r in off if r[5]]
    assert sum((-1) ** d for d in ess) == 1
    # the highest maximum has nothing older to die into: an infinite class
    maxima = [(int(d), int(s)) for d, s, pd, _ in grad if pd < 0 and d == 3]
    if maxima:
        assert any(r[5] and (int(r[0]), int(r[1])) == maxima[-1] for r in off)


def test_without_virtual_maximum_flat_grid_has_no_d2():
    """A one-voxel-thick grid has no tetrahedra: both options agree."""
    v = np.random.default_rng(51).random((1, 6, 7))
    on, gon = oracle.sandwich(v, virtual_max=True)
    off, goff = oracle.sandwich(v, virtual_max=False)
    assert _pairs(on) == _pairs(off) and gon == goff
    assert not any(r[0] == 2 and not r[5] for r in off)
