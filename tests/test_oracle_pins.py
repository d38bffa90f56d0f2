"""Pins of the oracle against what the paper and the mathematics fix.

Every function of ``oracle/`` is checked here against something other than
itself: closed forms, the paper's worked elevation case (Sec. 9.1), a
brute-force rank formula for the pairing, brute-force persistent Betti
numbers, two textbook union-find special cases, invariants at any size and
white-noise statistics.
"""
import json
import os
import zlib

import numpy as np
import pytest

import oracle
import synthfields as sf
from tests import bruteforce as bf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_field(rng, shape_xyz, kind):
    nx, ny, nz = shape_xyz
    n = nx * ny * nz
    if kind == "perm":
        return rng.permutation(n).astype(np.float32).reshape(nz, ny, nx)
    if kind == "ties":
        return rng.integers(0, 3, (nz, ny, nx)).astype(np.uint16)
    return rng.random((nz, ny, nx))


# ----------------------------------------------------------- closed forms

def _closed_form_counts(nx, ny, nz):
    """V, E, T, Tet of the Freudenthal triangulation by counting anchors: a
    chain simplex with largest offset o fits at prod_k (n_k - o_k) anchors."""
    n = (nx, ny, nz)

    def fits(o):
        return int(np.prod([n[k] - ((o >> k) & 1) for k in range(3)]))
    edges = sum(fits(o) for o in range(1, 8))
    # triangles: chains a < b of non-empty offsets (a a proper subset of b)
    tris = sum(fits(b) for b in range(1, 8) for a in range(1, 8) if a != b and a & b == a)
    tets = 6 * fits(7)
    return [nx * ny * nz, edges, tris, tets]


def test_simplex_counts_closed_form():
    cases = json.load(open(os.path.join(GOLDEN, "simplex_counts.json")))["cases"]
    for c in cases:
        assert c["counts"] == _closed_form_counts(*c["shape_xyz"])
        counts = oracle.simplex_counts(*c["shape_xyz"])
        assert list(counts) == c["counts"]
        assert counts[0] - counts[1] + counts[2] - counts[3] == 1   # chi of a cube


def test_simplex_ids_match_chain_definition():
    """Every id enumerated by the oracle names a chain simplex and vice versa."""
    for shape in [(2, 2, 2), (3, 2, 2), (3, 3, 3), (4, 2, 3)]:
        nx, ny, nz = shape
        brute = bf.freudenthal_simplices(shape)
        want = {(len(s) - 1, bf.simplex_id(shape, s)): s for s in brute}
        got = {}
        for dim, mult in enumerate((1, 7, 12, 6)):
            for sid in range(nx * ny * nz * mult):
                vs = oracle.simplex_vertices(shape, dim, sid)
                if vs is not None:
                    got[(dim, sid)] = frozenset(vs)
        assert got == want


# ------------------------------------------ Sec. 9.1: the elevation field

def test_elevation_single_bar():
    cases = json.load(open(os.path.join(GOLDEN, "elevation.json")))["cases"]
    for c in cases:
        for dt in (np.float32, np.uint16, np.float64):
            rows = oracle.pairsimplices(sf.ramp(c["shape_xyz"], dt))
            ess = [[int(r[0]), int(r[1])] for r in rows if r[5]]
            pairs = [r for r in rows if not r[5]]
            assert ess == c["essential"] and len(pairs) == len(c["pairs"])


def test_constant_field_is_ordered_by_id():
    """All values tie; the order is the vertex id order, a pure ramp in id."""
    for shape in [(3, 3, 3), (6, 5, 4)]:
        rows = oracle.pairsimplices(sf.constant(shape))
        assert [(int(r[0]), int(r[1]), int(r[5])) for r in rows] == [(0, 0, 1)]


# ------------------------------- brute-force pairing (pairing uniqueness)

@pytest.mark.parametrize("shape,kind,trials", [
    ((2, 2, 2), "perm", 60), ((2, 2, 2), "ties", 40), ((3, 2, 2), "perm", 12),
    ((3, 2, 2), "ties", 8), ((2, 2, 1), "perm", 10), ((3, 3, 1), "float", 6)])
def test_pairing_equals_rank_formula(shape, kind, trials):
    """All pairs (zero-persistence included) equal the rank-formula pairing."""
    rng = np.random.default_rng(zlib.crc32(repr((shape, kind)).encode()))
    for _ in range(trials):
        v = _rand_field(rng, shape, kind)
        keys = bf.vertex_keys(v)
        order = bf.lex_order(bf.freudenthal_simplices(shape), keys)
        want = set()
        paired = set()
        for i, j in bf.pairing_by_ranks(order):
            s, t = order[i], order[j]
            want.add((len(s) - 1, bf.simplex_id(shape, s), bf.simplex_id(shape, t)))
            paired |= {i, j}
        want_ess = {(len(order[i]) - 1, bf.simplex_id(shape, order[i]))
                    for i in range(len(order)) if i not in paired}
        rows = oracle.pairsimplices(v, keep_zero=True)
        got = {(int(r[0]), int(r[1]), int(r[2])) for r in rows if not r[5]}
        got_ess = {(int(r[0]), int(r[1])) for r in rows if r[5]}
        assert got == want and got_ess == want_ess


# ---------------------------------------- brute-force persistent Betti

@pytest.mark.parametrize("shape,kind,seed", [
    ((3, 3, 3), "perm", 0), ((3, 3, 3), "ties", 1), ((3, 3, 3), "float", 2),
    ((4, 3, 2), "perm", 3), ((3, 3, 3), "perm", 4)])
def test_persistent_betti(shape, kind, seed):
    """The vertex-level diagram reproduces every persistent Betti number."""
    rng = np.random.default_rng(seed)
    v = _rand_field(rng, shape, kind)
    beta, vrank = bf.persistent_betti(shape, v)
    rows = oracle.pairsimplices(v)
    assert np.array_equal(bf.diagram_betti(rows, vrank, len(vrank)), beta)


def test_interior_maximum_is_a_void():
    """3x3x3 with the centre on top: one D2 pair (boundary triangle, a tet of
    the centre) -- the centre's lower link is the whole 14-vertex sphere."""
    v = np.zeros((3, 3, 3), np.float32)
    v[1, 1, 1] = 10.0
    rows = oracle.pairsimplices(v)
    d2 = [r for r in rows if r[0] == 2 and not r[5]]
    assert len(d2) == 1 and d2[0][4] == 13


# ------------------------------------------- textbook union-find cases

@pytest.mark.parametrize("seed", range(6))
def test_union_find_special_cases(seed):
    """D0 = elder-rule union-find over all edges; D2 = union-find on the dual
    graph with a virtual maximum; both at the level of simplex ids."""
    rng = np.random.default_rng(100 + seed)
    for _ in range(12):
        shape = tuple(int(s) for s in rng.integers(1, 8, 3))
        v = _rand_field(rng, shape, ["perm", "ties", "float"][_ % 3])
        rows = oracle.pairsimplices(v)
        d0 = {(int(r[1]), int(r[2])) for r in rows if r[0] == 0}
        d2 = {(int(r[1]), int(r[2])) for r in rows if r[0] == 2 and not r[5]}
        k0 = {(int(r[1]), int(r[2])) for r in oracle.kruskal_d0(v)}
        k2 = {(int(r[1]), int(r[2])) for r in oracle.kruskal_d2(v)}
        assert d0 == k0 and d2 == k2


# ---------------------------------------------------------- invariants

def _chi_by_level(v):
    """chi(K_i) for every vertex level, by counting simplices directly."""
    nz, ny, nx = v.shape
    order = np.lexsort((np.arange(v.size), v.reshape(-1)))
    rank = np.empty(v.size, np.int64)
    rank[order] = np.arange(v.size)
    delta = np.zeros(v.size, np.int64)
    for dim, mult in enumerate((1, 7, 12, 6)):
        for sid in range(v.size * mult):
            vs = bf_vertices((nx, ny, nz), dim, sid)
            if vs is not None:
                delta[max(rank[list(vs)])] += (-1) ** dim
    return np.cumsum(delta), rank


def bf_vertices(shape, dim, sid):
    """Vertices of id ``sid`` from the documented convention (test-side)."""
    nx, ny, nz = shape
    mult = (1, 7, 12, 6)[dim]
    v, k = divmod(sid, mult)
    x, y, z = v % nx, (v // nx) % ny, v // (nx * ny)
    if dim == 0:
        offs = [0]
    elif dim == 1:
        offs = [0, k + 1]
    elif dim == 2:
        b, a = bf._TRI[k]
        offs = [0, a, b]
    else:
        a, b = bf._TET[k]
        offs = [0, a, b, 7]
    out = []
    for o in offs:
        p = (x + (o & 1), y + ((o >> 1) & 1), z + ((o >> 2) & 1))
        if p[0] >= nx or p[1] >= ny or p[2] >= nz:
            return None
        out.append(p[0] + nx * (p[1] + ny * p[2]))
    return out


@pytest.mark.parametrize("name,shape", [("noise", (12, 10, 9)), ("mixture", (14, 11, 9))])
def test_euler_characteristic_by_level(name, shape):
    """chi(K_i) = #D0 alive - #D1 alive + #D2 alive at every level i, and the
    pair counts satisfy |D0 finite| = #min - 1 with one essential class."""
    if name == "noise":
        v = sf.white_noise(shape, 7)
    else:
        v = sf.gaussian_mixture(shape, 6, 8, noise=1e-3)
    chi, rank = _chi_by_level(v)
    rows = oracle.pairsimplices(v)
    alive = np.zeros(v.size + 1, np.int64)
    for r in rows:
        b = rank[r[3]]
        d = v.size if r[5] else rank[r[4]]
        alive[b] += (-1) ** int(r[0])
        alive[d] -= (-1) ** int(r[0])
    assert np.array_equal(np.cumsum(alive)[: v.size], chi)
    ess = [r for r in rows if r[5]]
    assert len(ess) == 1 and ess[0][0] == 0 and rank[ess[0][1]] == 0
    assert chi[-1] == 1


def test_white_noise_minima_statistics():
    """For iid values, P(v is a minimum) = 1/(deg(v)+1): the count of minima
    (finite D0 pairs + 1) is within 5 sigma of the sum over vertices."""
    shape = (32, 32, 32)
    nx, ny, nz = shape
    v = sf.white_noise(shape, 11)
    deg = np.zeros((nz, ny, nx), np.int64)
    for o in range(1, 8):
        dx, dy, dz = o & 1, (o >> 1) & 1, (o >> 2) & 1
        deg[: nz - dz, : ny - dy, : nx - dx] += 1    # neighbour at +o
        deg[dz:, dy:, dx:] += 1                      # neighbour at -o
    p = 1.0 / (deg + 1.0)
    mean, sd = p.sum(), np.sqrt((p * (1 - p)).sum())
    rows = oracle.kruskal_d0(v)
    n_min = len(rows)          # finite pairs + the essential class
    assert abs(n_min - mean) < 5 * sd, (n_min, mean, sd)


# -------------------------------------------------------- input handling

def test_nan_rejected_and_signed_zero():
    v = np.zeros((3, 3, 3), np.float32)
    v[1, 1, 1] = np.nan
    with pytest.raises(ValueError):
        oracle.pairsimplices(v)
    a = sf.white_noise((4, 4, 3), 5)
    a[a < 0.3] = 0.0
    b = a.copy()
    b[a == 0.0] = -0.0
    assert np.array_equal(oracle.pairsimplices(a), oracle.pairsimplices(b))


def test_dtype_invariance():
    """Only the order matters: u16, f32 and f64 with the same ranks agree."""
    rng = np.random.default_rng(3)
    q = rng.integers(0, 50, (5, 6, 7))
    outs = [oracle.pairsimplices(q.astype(dt)) for dt in (np.uint16, np.float32, np.float64)]
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
