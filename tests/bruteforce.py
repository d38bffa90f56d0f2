"""Brute-force checks of persistence on tiny grids, written from definitions.

Used only by tests to pin the oracle; shares no code with it.

- Freudenthal simplices are enumerated from their order-theoretic definition:
  a set of grid points is a simplex iff it is totally ordered by the
  componentwise order and its maximum minus its minimum lies in {0,1}^3
  (Sec. 2.1: each cube is split into 6 tetrahedra along its main diagonal).
- The lexicographic filtration follows Sec. 2.2 (decreasing vertex keys,
  compared lexicographically, a face before its cofaces), with keys
  (value, vertex id) (Sec. 2.1, symbolic perturbation).
- The pairing is read off ranks of submatrices of the boundary matrix (the
  pairing uniqueness lemma: simplices i < j are paired iff
  r(i,j) - r(i+1,j) - r(i,j-1) + r(i+1,j-1) = 1, where r(i,j) is the GF(2)
  rank of the rows >= i and columns <= j), with no column reduction.
- Persistent Betti numbers of the lower-star filtration at vertex levels are
  computed from the definition beta_p^{i,j} = dim Z_p(K_i) - dim(Z_p(K_i) ∩
  B_p(K_j)) with GF(2) ranks (Sec. 2.4).
"""
from __future__ import annotations

import itertools

import numpy as np


def vertex_keys(values: np.ndarray):
    """Key of vertex v = (value, v); -0.0 equals +0.0 (numeric comparison)."""
    flat = values.reshape(-1)
    return [(float(flat[v]) if flat.dtype.kind == "f" else int(flat[v]), v)
            for v in range(flat.size)]


def freudenthal_simplices(shape_xyz):
    """All simplices as frozensets of vertex ids, by the chain definition."""
    nx, ny, nz = shape_xyz

    def vid(p):
        return p[0] + nx * (p[1] + ny * p[2])

    out = set()
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                cube = [(x + dx, y + dy, z + dz) for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)
                        if x + dx < nx and y + dy < ny and z + dz < nz]
                for k in range(1, 5):
                    for pts in itertools.combinations(cube, k):
                        pts = sorted(pts, key=lambda p: sum(p))
                        chain = all(all(a <= b for a, b in zip(pts[i], pts[i + 1]))
                                    for i in range(len(pts) - 1))
                        if chain:
                            out.add(frozenset(vid(p) for p in pts))
    return sorted(out, key=lambda s: (len(s), sorted(s)))


def lex_order(simplices, keys):
    def k(s):
        return tuple(sorted((keys[v] for v in s), reverse=True))
    # a proper prefix sorts first because Python compares shorter tuples first
    return sorted(simplices, key=k)


class GF2Basis:
    """Incremental GF(2) row-echelon basis over Python-int bit vectors."""

    def __init__(self):
        self.piv = {}

    def add(self, vec: int) -> bool:
        while vec:
            h = vec.bit_length() - 1
            if h in self.piv:
                vec ^= self.piv[h]
            else:
                self.piv[h] = vec
                return True
        return False

    @property
    def rank(self):
        return len(self.piv)


def boundary_columns(order):
    """Column j = bit vector over positions of the facets of order[j]."""
    pos = {s: i for i, s in enumerate(order)}
    cols = []
    for s in order:
        v = 0
        if len(s) > 1:
            for u in s:
                v |= 1 << pos[s - {u}]
        cols.append(v)
    return cols


def pairing_by_ranks(order):
    """Set of (i, j) position pairs, from the rank formula only."""
    n = len(order)
    cols = boundary_columns(order)
    # r[i][j+1] = rank of rows >= i, columns <= j ; r[i][0] = 0; r[n][*] = 0
    r = np.zeros((n + 1, n + 1), dtype=np.int64)
    for i in range(n):
        mask = ~((1 << i) - 1)
        b = GF2Basis()
        for j in range(n):
            b.add(cols[j] & mask)
            r[i, j + 1] = b.rank
    pairs = set()
    for i in range(n):
        for j in range(i + 1, n):
            # columns <= j -> index j+1 ; columns <= j-1 -> index j
            if r[i, j + 1] - r[i + 1, j + 1] - r[i, j] + r[i + 1, j] == 1:
                pairs.add((i, j))
    return pairs


def _rank(vectors):
    b = GF2Basis()
    for v in vectors:
        b.add(v)
    return b.rank


def persistent_betti(shape_xyz, values):
    """beta[p][i][j] for vertex levels i <= j of the lower-star filtration.

    K_i = all simplices whose maximum vertex has rank <= i."""
    keys = vertex_keys(values)
    simp = freudenthal_simplices(shape_xyz)
    nv = len(keys)
    vrank = {v: r for r, v in enumerate(sorted(range(nv), key=lambda v: keys[v]))}
    level = {s: max(vrank[v] for v in s) for s in simp}
    by_dim = [[s for s in simp if len(s) == p + 1] for p in range(4)]
    index = [{s: k for k, s in enumerate(by_dim[p])} for p in range(4)]

    def bvec(s):
        p = len(s) - 1
        v = 0
        for u in s:
            v |= 1 << index[p - 1][s - {u}]
        return v

    beta = np.zeros((3, nv, nv), dtype=np.int64)
    for p in range(3):
        for i in range(nv):
            cp_i = [s for s in by_dim[p] if level[s] <= i]
            mask_i = 0
            for s in cp_i:
                mask_i |= 1 << index[p][s]
            z_i = len(cp_i) - (_rank([bvec(s) for s in cp_i]) if p > 0 else 0)
            for j in range(i, nv):
                cols = [bvec(s) for s in by_dim[p + 1] if level[s] <= j]
                # dim(B_p(K_j) ∩ C_p(K_i)) = rank(all) - rank(rows outside K_i)
                inter = _rank(cols) - _rank([c & ~mask_i for c in cols])
                beta[p, i, j] = z_i - inter
    return beta, vrank


def diagram_betti(rows, vrank, nv):
    """beta[p][i][j] implied by a diagram: pairs with b <= i < d plus the
    essential classes born at b <= i (levels are vertex ranks)."""
    beta = np.zeros((3, nv, nv), dtype=np.int64)
    for r in rows:
        p, ess, bv, dv = int(r[0]), int(r[5]), int(r[3]), int(r[4])
        if p > 2:
            continue
        b = vrank[bv]
        d = nv if ess else vrank[dv]
        for i in range(b, nv):
            for j in range(i, nv):
                if j < d:
                    beta[p, i, j] += 1
    return beta


# The project's simplex id convention (documented in include/dms.h): an
# anchor v (the componentwise-minimum corner) and offset bitmasks from it.
_TRI = [(3, 1), (3, 2), (5, 1), (5, 4), (6, 2), (6, 4), (7, 1), (7, 2), (7, 3), (7, 4),
        (7, 5), (7, 6)]
_TET = [(1, 3), (1, 5), (2, 3), (2, 6), (4, 5), (4, 6)]


def simplex_id(shape_xyz, s):
    """Id of the simplex with vertex set ``s`` under the documented scheme."""
    nx, ny, nz = shape_xyz
    pts = [(v % nx, (v // nx) % ny, v // (nx * ny)) for v in s]
    a = tuple(min(p[k] for p in pts) for k in range(3))
    anchor = a[0] + nx * (a[1] + ny * a[2])
    offs = sorted(((p[0] - a[0]) | ((p[1] - a[1]) << 1) | ((p[2] - a[2]) << 2)) for p in pts)
    offs = [o for o in offs if o]
    if len(s) == 1:
        return anchor
    if len(s) == 2:
        return 7 * anchor + offs[0] - 1
    if len(s) == 3:
        lo, hi = sorted(offs, key=lambda o: bin(o).count("1"))
        return 12 * anchor + _TRI.index((hi, lo))
    one = [o for o in offs if bin(o).count("1") == 1][0]
    two = [o for o in offs if bin(o).count("1") == 2][0]
    return 6 * anchor + _TET.index((one, two))
