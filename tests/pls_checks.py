"""The kernels' lower-star code, built for the host, against the oracle.

    python -m tests.pls_checks <directory holding dms_common.cuh>

``build_harness`` compiles ``tests/host/pls_host.cc`` against the
``dms_common.cuh`` of a directory (the kernels' ``csrc/``, or a copy with a
planted mistake); ``Harness`` runs its ProcessLowerStars, star view and order
keys with the star tables the library builds (``dms_star_tables``).  The
checks compare them with the oracle's gradient star by star, and with the
order of the values.  As a program it runs a compact set of them and exits 0
when all pass, 1 when one fails (a crash ends it with its own status).
"""
import ctypes
import os
import subprocess
import sys
import tempfile

import numpy as np

import oracle
from tests import bruteforce as bf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2206_13932_gb300", "csrc")
CUDA_INCLUDE = "/usr/local/cuda/include"
K_NONE, K_HEAD = 63, 62


def build_harness(include_dir, out_path):
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-Wall",
                           "-Wno-attributes", "-Wno-unknown-pragmas", f"-I{include_dir}",
                           f"-I{CUDA_INCLUDE}", os.path.join(ROOT, "tests", "host", "pls_host.cc"),
                           "-o", out_path])
    return out_path


class Harness:
    def __init__(self, so_path):
        import paper_2206_13932_gb300 as dms
        lib = dms.load(build_if_missing=True)
        lib.dms_star_tables.restype = ctypes.c_int64
        lib.dms_star_tables.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        h = ctypes.CDLL(so_path)
        h.harness_tables_size.restype = ctypes.c_int64
        h.harness_pls.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p,
                                  ctypes.c_void_p]
        h.harness_layout.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        h.harness_load_star.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                        ctypes.c_void_p]
        h.harness_key_f32.argtypes = [ctypes.c_float]
        h.harness_key_f32.restype = ctypes.c_uint64
        h.harness_key_f64.argtypes = [ctypes.c_double]
        h.harness_key_f64.restype = ctypes.c_uint64
        h.harness_nan_f32.argtypes = [ctypes.c_float]
        h.harness_nan_f64.argtypes = [ctypes.c_double]
        size = lib.dms_star_tables(None, 0)
        assert size == h.harness_tables_size() > 0, "star table layouts differ"
        self.tables = ctypes.create_string_buffer(int(size))
        assert lib.dms_star_tables(self.tables, size) == size
        lay = (ctypes.c_int64 * 186)()
        h.harness_layout(self.tables, lay)
        lay = list(lay)
        self.offs = [tuple(lay[3 * n:3 * n + 3]) for n in range(14)]
        self.tri_v = [tuple(lay[42 + 2 * s:44 + 2 * s]) for s in range(36)]
        self.tet_v = [tuple(lay[114 + 3 * t:117 + 3 * t]) for t in range(24)]
        self.h = h

    # ---- one lower star
    def star_cells(self, shape, v, keys):
        """Lower mask, ranks and the vertex set of every star cell of vertex v,
        from the order (value, id)."""
        nx, ny, nz = shape
        x, y, z = v % nx, (v // nx) % ny, v // (nx * ny)
        nb = []
        for dx, dy, dz in self.offs:
            p = (x + dx, y + dy, z + dz)
            ok = 0 <= p[0] < nx and 0 <= p[1] < ny and 0 <= p[2] < nz
            nb.append(p[0] + nx * (p[1] + ny * p[2]) if ok else None)
        lower = [n for n in range(14) if nb[n] is not None and keys[nb[n]] < keys[v]]
        L = sum(1 << n for n in lower)
        rank = [0] * 14
        for r, n in enumerate(sorted(lower, key=lambda n: keys[nb[n]])):
            rank[n] = r
        edge = {n: frozenset((v, nb[n])) for n in lower}
        tri = {s: frozenset((v, nb[a], nb[b])) for s, (a, b) in enumerate(self.tri_v)
               if L >> a & 1 and L >> b & 1}
        tet = {t: frozenset((v, nb[a], nb[b], nb[c])) for t, (a, b, c) in enumerate(self.tet_v)
               if L >> a & 1 and L >> b & 1 and L >> c & 1}
        return L, rank, edge, tri, tet, nb

    def library_star(self, shape, v, keys):
        """Critical cells and pairs of the library's ProcessLowerStars."""
        L, rank, edge, tri, tet, _ = self.star_cells(shape, v, keys)
        out = (ctypes.c_int64 * 10)()
        self.h.harness_pls(self.tables, L, (ctypes.c_uint8 * 14)(*rank), out)
        crit_e, crit_t, crit_h, is_min = (int(out[k]) & (2 ** 64 - 1) for k in range(4))
        w = [int(x) & (2 ** 64 - 1) for x in out[4:10]]
        tpair = [(w[h // 10] >> (6 * (h % 10))) & 63 for h in range(24)]
        epair = [((w[2] >> (24 + 6 * n)) if n < 6 else (w[3] >> (6 * (n - 6)))) & 63
                 for n in range(14)]
        crit = {frozenset((v,))} if is_min else set()
        crit |= {edge[n] for n in edge if crit_e >> n & 1}
        crit |= {tri[s] for s in tri if crit_t >> s & 1}
        crit |= {tet[t] for t in tet if crit_h >> t & 1}
        pairs = set()
        for n in edge:
            if epair[n] == K_HEAD:
                pairs.add((frozenset((v,)), edge[n]))
            elif epair[n] != K_NONE:
                pairs.add((edge[n], tri[epair[n]]))
        for t in tet:
            if tpair[t] != K_NONE:
                pairs.add((tri[tpair[t]], tet[t]))
        return crit, pairs

    def load_star(self, values, shape, v):
        """(present, lower, descent, ranks) of the kernels' star view."""
        code = {np.dtype(np.uint16): 0, np.dtype(np.float32): 1, np.dtype(np.float64): 2}
        flat = np.ascontiguousarray(values).reshape(-1)
        out = (ctypes.c_int64 * 17)()
        nx, ny, nz = shape
        self.h.harness_load_star(self.tables, code[flat.dtype], flat.ctypes.data, nx, ny, nz, v,
                                 out)
        return int(out[0]), int(out[1]), int(out[2]), [int(out[3 + n]) for n in range(14)]


_CELLS = {}


def cells_of(shape):
    """(dim, id) -> vertex set, from the brute-force chain definition."""
    if shape not in _CELLS:
        _CELLS[shape] = {(len(s) - 1, bf.simplex_id(shape, s)): s
                         for s in bf.freudenthal_simplices(shape)}
    return _CELLS[shape]


def oracle_stars(values, vertices=None):
    """Per vertex: critical cells and pairs of the oracle's gradient in its
    lower star (only the stars of ``vertices`` when given)."""
    nz, ny, nx = values.shape
    shape = (nx, ny, nz)
    keys = bf.vertex_keys(values)
    cells = cells_of(shape)
    crit, pairs = {}, {}
    for d, sid, pd, pid in oracle.gradient(values):
        s = cells[(int(d), int(sid))]
        if vertices is not None and not any(u in s for u in vertices):
            continue
        top = max(s, key=lambda u: keys[u])
        if pd < 0:
            crit.setdefault(top, set()).add(s)
        elif pd > d:
            pairs.setdefault(top, set()).add((s, cells[(int(pd), int(pid))]))
    return shape, keys, crit, pairs


def check_field(hv, values, vertices=None):
    """Every lower star (or those of ``vertices``) of the library against the
    oracle; returns the oracle's critical cells per vertex."""
    shape, keys, crit, pairs = oracle_stars(values, vertices)
    for v in (range(len(keys)) if vertices is None else vertices):
        got_crit, got_pairs = hv.library_star(shape, v, keys)
        assert got_crit == crit.get(v, set()), ("critical cells", v)
        assert got_pairs == pairs.get(v, set()), ("pairs", v)
    return crit


def check_star_view(hv, values):
    """The kernels' star view against the order (value, id)."""
    nz, ny, nx = values.shape
    shape = (nx, ny, nz)
    keys = bf.vertex_keys(values)
    for vid in range(values.size):
        present, lower, descent, ranks = hv.load_star(values, shape, vid)
        L, rank, _, _, _, nb = hv.star_cells(shape, vid, keys)
        want_present = sum(1 << n for n in range(14) if nb[n] is not None)
        assert present == want_present and lower == L, ("lower links", vid)
        assert [ranks[n] for n in range(14) if L >> n & 1] == \
            [rank[n] for n in range(14) if L >> n & 1], ("ranks", vid)
        lowest = [n for n in range(14) if L >> n & 1 and rank[n] == 0]
        assert descent == (lowest[0] if lowest else 0xF), ("descent", vid)


def random_field(rng, shape, kind):
    nx, ny, nz = shape
    if kind == "float":
        return rng.random((nz, ny, nx)) - 0.5
    if kind == "ties":
        return rng.integers(0, 3, (nz, ny, nx)).astype(np.uint16)
    if kind == "ties64":
        return rng.integers(0, 3, (nz, ny, nx)).astype(np.float64)
    if kind == "signed":
        pool = np.array([-0.0, 0.0, -1.5, 1.5, np.inf, -np.inf, 2.0], dtype=np.float32)
        return pool[rng.integers(0, len(pool), (nz, ny, nx))]
    return (rng.permutation(nx * ny * nz) - nx * ny * nz // 2).astype(np.float32) \
        .reshape(nz, ny, nx)


def main(include_dir):
    with tempfile.TemporaryDirectory() as tmp:
        hv = Harness(build_harness(include_dir, os.path.join(tmp, "libplshost.so")))
        rng = np.random.default_rng(3)
        failed = []
        try:
            for shape in [(3, 3, 3), (4, 3, 3), (3, 4, 2), (4, 4, 3), (5, 3, 1)]:
                for kind in ("float", "ties", "ties64", "perm", "signed"):
                    for rep in range(6):
                        v = random_field(rng, shape, kind)
                        if rep == 0:
                            check_star_view(hv, v)
                        check_field(hv, v)
            for _ in range(1024):                     # random lower masks of an interior star
                m = int(rng.integers(0, 1 << 14))
                v = rng.random(27) + 2.0
                v[13] = 1.5
                for n, (dx, dy, dz) in enumerate(hv.offs):
                    if m >> n & 1:
                        v[(1 + dx) + 3 * ((1 + dy) + 3 * (1 + dz))] = rng.random()
                check_field(hv, v.reshape(3, 3, 3), vertices=[13])
        except AssertionError as e:
            failed.append(str(e))
        for f in failed:
            print(f)
        return 1 if failed else 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1]))
