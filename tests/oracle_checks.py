"""A compact run of the oracle's pins against an oracle package at any path.

    python -m tests.oracle_checks <directory holding an oracle/ package>

Exit status 0 when every check passes, 1 when one fails (a crash of the
oracle ends the process with its own status).  ``tests/test_oracle_mutants.py``
runs it on copies of the oracle with one planted mistake each.  The checks
are the independent ones of ``test_oracle_pins.py`` and
``test_oracle_sandwich.py``, on small cases: the id scheme against the chain
definition, the pairing against the rank formula, persistent Betti numbers,
the union-find special cases, the elevation bar, the sandwich's steps against
the standard reduction, generator cycles, the invariants of the option
without the virtual maximum, and the fast-mode reduction against the rank
formula and the textbook mode.
"""
import importlib.util
import os
import sys

import numpy as np

from tests import bruteforce as bf


def load(directory):
    path = os.path.join(directory, "oracle", "__init__.py")
    spec = importlib.util.spec_from_file_location("oracle_under_test", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _field(rng, shape, kind):
    nx, ny, nz = shape
    n = nx * ny * nz
    if kind == "perm":     # signed values: negative floats must order too
        return (rng.permutation(n) - n // 2).astype(np.float32).reshape(nz, ny, nx)
    if kind == "ties":
        return rng.integers(0, 3, (nz, ny, nx)).astype(np.uint16)
    return (rng.random((nz, ny, nx)) - 0.5)


def check_ids(orc):
    for shape in [(2, 2, 2), (3, 2, 2)]:
        nx, ny, nz = shape
        want = {(len(s) - 1, bf.simplex_id(shape, s)): s for s in bf.freudenthal_simplices(shape)}
        got = {}
        for dim, mult in enumerate((1, 7, 12, 6)):
            for sid in range(nx * ny * nz * mult):
                vs = orc.simplex_vertices(shape, dim, sid)
                if vs is not None:
                    got[(dim, sid)] = frozenset(vs)
        assert got == want, "simplex ids"


def check_rank_formula(orc):
    rng = np.random.default_rng(5)
    for shape, kind, trials in [((2, 2, 2), "perm", 10), ((3, 2, 2), "ties", 4),
                                ((2, 2, 2), "float", 4)]:
        for _ in range(trials):
            v = _field(rng, shape, kind)
            order = bf.lex_order(bf.freudenthal_simplices(shape), bf.vertex_keys(v))
            want, paired = set(), set()
            for i, j in bf.pairing_by_ranks(order):
                want.add((len(order[i]) - 1, bf.simplex_id(shape, order[i]),
                          bf.simplex_id(shape, order[j])))
                paired |= {i, j}
            rows = orc.pairsimplices(v, keep_zero=True)
            assert {(int(r[0]), int(r[1]), int(r[2])) for r in rows if not r[5]} == want, \
                "rank formula"
            assert {(int(r[0]), int(r[1])) for r in rows if r[5]} == \
                {(len(order[i]) - 1, bf.simplex_id(shape, order[i]))
                 for i in range(len(order)) if i not in paired}, "rank formula (infinite)"


def check_betti(orc):
    rng = np.random.default_rng(6)
    v = _field(rng, (3, 3, 3), "perm")
    beta, vrank = bf.persistent_betti((3, 3, 3), v)
    assert np.array_equal(bf.diagram_betti(orc.pairsimplices(v), vrank, len(vrank)), beta), \
        "persistent Betti"


def _pairs(rows, dim=None):
    return {(int(r[0]), int(r[1]), int(r[2]), int(r[5])) for r in rows
            if dim is None or int(r[0]) == dim}


def check_union_find(orc):
    rng = np.random.default_rng(7)
    for shape in [(5, 4, 3), (4, 4, 4)]:
        v = _field(rng, shape, "float")
        rows = orc.pairsimplices(v)
        assert _pairs(orc.kruskal_d0(v)) == _pairs(rows, 0), "D0 by union-find"
        assert _pairs(orc.kruskal_d2(v)) == {p for p in _pairs(rows, 2) if not p[3]}, \
            "D2 by union-find"


def check_elevation(orc):
    nx, ny, nz = 5, 4, 3
    z, y, x = np.meshgrid(range(nz), range(ny), range(nx), indexing="ij")
    rows = orc.pairsimplices((x + y + z).astype(np.float32))
    assert [(int(r[0]), int(r[1]), int(r[5])) for r in rows] == [(0, 0, 1)], "elevation"


def check_sandwich(orc):
    rng = np.random.default_rng(8)
    for shape, kind in [((4, 3, 3), "perm"), ((4, 3, 3), "ties"), ((3, 4, 2), "float")]:
        v = _field(rng, shape, kind)
        rows, gens = orc.sandwich(v)
        assert _pairs(rows) == _pairs(orc.pairsimplices(v)), "sandwich = reduction"
        assert set(gens) == {(int(r[1]), int(r[2])) for r in rows if r[0] == 1 and not r[5]}


def check_generators(orc):
    rng = np.random.default_rng(9)
    v = _field(rng, (3, 3, 3), "perm")
    keys = bf.vertex_keys(v)
    cells = {(len(s) - 1, bf.simplex_id((3, 3, 3), s)): s
             for s in bf.freudenthal_simplices((3, 3, 3))}

    def lex(s):
        return tuple(sorted((keys[u] for u in s), reverse=True))
    edges = sorted((s for s in cells.values() if len(s) == 2), key=lex)
    eidx = {s: i for i, s in enumerate(edges)}
    tris = sorted((s for s in cells.values() if len(s) == 3), key=lex)
    _, gens = orc.sandwich(v)
    assert gens, "no D1 pair to check"
    for (birth, death), cycle in gens.items():
        cyc = [cells[(1, e)] for e in cycle]
        deg = {}
        for e in cyc:
            for u in e:
                deg[u] = deg.get(u, 0) ^ 1
        assert not any(deg.values()), "generator not a cycle"
        assert max(cyc, key=lex) == cells[(1, birth)], "generator top"
        t = cells[(2, death)]
        basis = bf.GF2Basis()
        for u in tris:
            if lex(u) >= lex(t):
                break
            basis.add(sum(1 << eidx[u - {w}] for w in u))
        vec = sum(1 << eidx[e] for e in cyc) ^ sum(1 << eidx[t - {w}] for w in t)
        while vec and (vec.bit_length() - 1) in basis.piv:
            vec ^= basis.piv[vec.bit_length() - 1]
        assert vec == 0, "generator not homologous"


def check_without_virtual_max(orc):
    rng = np.random.default_rng(10)
    for shape in [(8, 7, 6), (7, 7, 7)]:     # large enough to hold interior maxima
        v = _field(rng, shape, "float")
        on, _ = orc.sandwich(v, virtual_max=True)
        off, _ = orc.sandwich(v, virtual_max=False)
        assert _pairs(on, 0) == _pairs(off, 0), "D0 changed"
        assert sum((-1) ** int(r[0]) for r in off if r[5]) == 1, "infinite classes"
        grad = orc.gradient(v)
        maxima = [(int(d), int(s)) for d, s, pd, _ in grad if pd < 0 and d == 3]
        assert maxima, "no maximum to check"
        assert any(r[5] and (int(r[0]), int(r[1])) == maxima[-1] for r in off), \
            "highest maximum"


def check_fast(orc):
    """The fast-mode reduction against the rank formula and the textbook mode."""
    rng = np.random.default_rng(11)
    for shape, kind, trials in [((2, 2, 2), "perm", 8), ((3, 2, 2), "ties", 4)]:
        for _ in range(trials):
            v = _field(rng, shape, kind)
            order = bf.lex_order(bf.freudenthal_simplices(shape), bf.vertex_keys(v))
            want, paired = set(), set()
            for i, j in bf.pairing_by_ranks(order):
                want.add((len(order[i]) - 1, bf.simplex_id(shape, order[i]),
                          bf.simplex_id(shape, order[j])))
                paired |= {i, j}
            rows = orc.fastpairs(v, keep_zero=True)
            assert {(int(r[0]), int(r[1]), int(r[2])) for r in rows if not r[5]} == want, \
                "fast mode: rank formula"
            assert {(int(r[0]), int(r[1])) for r in rows if r[5]} == \
                {(len(order[i]) - 1, bf.simplex_id(shape, order[i]))
                 for i in range(len(order)) if i not in paired}, "fast mode: infinite"
    for shape, kind in [((6, 5, 4), "float"), ((5, 5, 4), "ties")]:
        v = _field(rng, shape, kind)
        full = {tuple(int(x) for x in r[:6]) for r in orc.pairsimplices(v)}
        assert {tuple(int(x) for x in r[:6]) for r in orc.fastpairs(v)} == full, \
            "fast mode = textbook"


CHECKS = [check_ids, check_rank_formula, check_betti, check_union_find, check_elevation,
          check_sandwich, check_generators, check_without_virtual_max, check_fast]


def main(directory):
    orc = load(directory)
    failed = []
    for check in CHECKS:
        try:
            check(orc)
        except Exception as e:   # a failing pin, or an oracle error
            failed.append(f"{check.__name__}: {e}")
    for f in failed:
        print(f)
    return 1 if failed else 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1]))
