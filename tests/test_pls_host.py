"""The library's ProcessLowerStars source, run on the host, against the oracle.

``tests/host/pls_host.cc`` compiles ``csrc/dms_common.cuh`` (the code the
kernels run) for the host, with the star tables the library builds
(``dms_star_tables``).  For every lower star of small random fields, with and
without ties, and for every lower-link mask of an interior vertex, its
critical cells and its pairs must equal the oracle's gradient (Alg. 2,
``oracle/sandwich.c``) restricted to that lower star, simplex for simplex.
No GPU is involved: this pins the logic of the gradient kernels; the GPU
parity tests pin their device build.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from tests import bruteforce as bf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INCLUDE = "/usr/local/cuda/include"
K_NONE, K_HEAD = 63, 62


@pytest.fixture(scope="module")
def star(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.isdir(CUDA_INCLUDE):
        pytest.skip("needs g++ and the CUDA headers")
    import paper_2206_13932_gb300 as dms
    lib = dms.load(build_if_missing=True)
    lib.dms_star_tables.restype = ctypes.c_int64
    lib.dms_star_tables.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    out = str(tmp_path_factory.mktemp("plshost") / "libplshost.so")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-Wall",
                           "-Wno-attributes", "-Wno-unknown-pragmas", f"-I{CUDA_INCLUDE}",
                           os.path.join(ROOT, "tests", "host", "pls_host.cc"), "-o", out])
    h = ctypes.CDLL(out)
    h.harness_tables_size.restype = ctypes.c_int64
    h.harness_pls.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]
    h.harness_layout.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    size = lib.dms_star_tables(None, 0)
    assert size == h.harness_tables_size() > 0
    tables = ctypes.create_string_buffer(int(size))
    assert lib.dms_star_tables(tables, size) == size
    lay = (ctypes.c_int64 * 186)()
    h.harness_layout(tables, lay)
    lay = list(lay)
    offs = [tuple(lay[3 * n:3 * n + 3]) for n in range(14)]
    tri_v = [tuple(lay[42 + 2 * s:44 + 2 * s]) for s in range(36)]
    tet_v = [tuple(lay[114 + 3 * t:117 + 3 * t]) for t in range(24)]
    return h, tables, offs, tri_v, tet_v


def _decode(w):
    """Pairs packed by the lower-star code (the layout of GradRec)."""
    w = [int(x) & (2 ** 64 - 1) for x in w]
    tpair = [(w[0 if h < 10 else 1 if h < 20 else 2] >> (6 * (h - 10 * (h // 10)))) & 63
             for h in range(24)]
    epair = [((w[2] >> (24 + 6 * n)) if n < 6 else (w[3] >> (6 * (n - 6)))) & 63
             for n in range(14)]
    return tpair, epair


def _star_cells(star_layout, shape, v, keys):
    """Lower mask, ranks and the vertex set of every star cell of vertex v."""
    _, _, offs, tri_v, tet_v = star_layout
    nx, ny, nz = shape
    x, y, z = v % nx, (v // nx) % ny, v // (nx * ny)
    nb = []
    for dx, dy, dz in offs:
        p = (x + dx, y + dy, z + dz)
        ok = 0 <= p[0] < nx and 0 <= p[1] < ny and 0 <= p[2] < nz
        nb.append(p[0] + nx * (p[1] + ny * p[2]) if ok else None)
    lower = [n for n in range(14) if nb[n] is not None and keys[nb[n]] < keys[v]]
    L = sum(1 << n for n in lower)
    rank = [0] * 14
    for r, n in enumerate(sorted(lower, key=lambda n: keys[nb[n]])):
        rank[n] = r
    edge = {n: frozenset((v, nb[n])) for n in lower}
    tri = {s: frozenset((v, nb[a], nb[b])) for s, (a, b) in enumerate(tri_v)
           if L >> a & 1 and L >> b & 1}
    tet = {t: frozenset((v, nb[a], nb[b], nb[c])) for t, (a, b, c) in enumerate(tet_v)
           if L >> a & 1 and L >> b & 1 and L >> c & 1}
    return L, rank, edge, tri, tet


def _library_star(star_layout, shape, v, keys):
    h, tables = star_layout[0], star_layout[1]
    L, rank, edge, tri, tet = _star_cells(star_layout, shape, v, keys)
    out = (ctypes.c_int64 * 10)()
    h.harness_pls(tables, L, (ctypes.c_uint8 * 14)(*rank), out)
    crit_e, crit_t, crit_h, is_min = (int(out[k]) & (2 ** 64 - 1) for k in range(4))
    tpair, epair = _decode(out[4:10])
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


_CELLS = {}


def _cells(shape):
    """(dim, id) -> vertex set, from the brute-force chain definition."""
    if shape not in _CELLS:
        _CELLS[shape] = {(len(s) - 1, bf.simplex_id(shape, s)): s
                         for s in bf.freudenthal_simplices(shape)}
    return _CELLS[shape]


def _oracle_stars(values, vertices=None):
    """Per vertex: critical cells and pairs of the oracle's gradient in its
    lower star."""
    nz, ny, nx = values.shape
    shape = (nx, ny, nz)
    keys = bf.vertex_keys(values)
    cells = _cells(shape)
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


def _check_field(star_layout, values, vertices=None):
    """Compares every lower star (or those of ``vertices``); returns the
    oracle's critical cells per vertex."""
    shape, keys, crit, pairs = _oracle_stars(values, vertices)
    for v in (range(len(keys)) if vertices is None else vertices):
        got_crit, got_pairs = _library_star(star_layout, shape, v, keys)
        assert got_crit == crit.get(v, set()), v
        assert got_pairs == pairs.get(v, set()), v
    return crit


@pytest.mark.parametrize("kind", ["float", "ties", "perm"])
def test_every_lower_star_of_random_fields(star, kind):
    rng = np.random.default_rng({"float": 1, "ties": 2, "perm": 3}[kind])
    for shape in [(3, 3, 3), (4, 3, 3), (3, 4, 2), (2, 2, 2), (5, 3, 1)]:
        for _ in range(6):
            nx, ny, nz = shape
            if kind == "float":
                v = rng.random((nz, ny, nx))
            elif kind == "ties":
                v = rng.integers(0, 3, (nz, ny, nx)).astype(np.uint16)
            else:
                v = rng.permutation(nx * ny * nz).astype(np.float32).reshape(nz, ny, nx)
            _check_field(star, v)


def test_every_lower_link_mask_of_an_interior_vertex(star):
    """All 2^14 lower masks of the centre of a 3x3x3 grid, each with random
    values (so random ranks) on its lower and upper neighbours.  The
    classification's table of PL-regular masks (``dms_regular_table``) must
    mark exactly the masks whose lower star has no critical cell in the
    oracle's gradient (Sec. 2.6: critical cells lie only in lower stars of PL
    critical points)."""
    import paper_2206_13932_gb300 as dms
    lib = dms.load()
    lib.dms_regular_table.restype = ctypes.c_int64
    lib.dms_regular_table.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    words = lib.dms_regular_table(None, 0)
    assert words == (1 << 14) // 32
    table = (ctypes.c_uint32 * words)()
    assert lib.dms_regular_table(table, words) == words
    rng = np.random.default_rng(7)
    _, _, offs, _, _ = star
    centre = 13
    link_ids = [(1 + dx) + 3 * ((1 + dy) + 3 * (1 + dz)) for dx, dy, dz in offs]
    regular = 0
    for m in range(1 << 14):
        v = rng.random(27) + 2.0                     # everything above the centre
        v[centre] = 1.5
        for n in range(14):
            if m >> n & 1:
                v[link_ids[n]] = rng.random()        # below the centre
        crit = _check_field(star, v.reshape(3, 3, 3), vertices=[centre])
        is_regular = not crit.get(centre)
        assert bool(table[m >> 5] >> (m & 31) & 1) == is_regular, m
        regular += is_regular
    assert 0 < regular < 1 << 14


def _harness_extra(star):
    h = star[0]
    h.harness_load_star.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p]
    h.harness_key_f32.argtypes = [ctypes.c_float]
    h.harness_key_f32.restype = ctypes.c_uint64
    h.harness_key_f64.argtypes = [ctypes.c_double]
    h.harness_key_f64.restype = ctypes.c_uint64
    h.harness_nan_f32.argtypes = [ctypes.c_float]
    h.harness_nan_f64.argtypes = [ctypes.c_double]
    return h


@pytest.mark.parametrize("dtype", [np.uint16, np.float32, np.float64])
def test_star_view_follows_the_vertex_order(star, dtype):
    """load_star (lower links, their ranks, the descent link) against the
    order by (value, vertex id) of Sec. 2.1, with heavy ties and signed zeros."""
    h = _harness_extra(star)
    _, tables, offs, _, _ = star
    rng = np.random.default_rng(11)
    code = {np.uint16: 0, np.float32: 1, np.float64: 2}[dtype]
    for shape in [(3, 3, 3), (5, 4, 3), (4, 1, 6), (1, 1, 5)]:
        nx, ny, nz = shape
        for _ in range(4):
            if dtype == np.uint16:
                v = rng.integers(0, 3, (nz, ny, nx)).astype(np.uint16)
            else:
                pool = np.array([-0.0, 0.0, -1.5, 1.5, np.inf, -np.inf, 2.0], dtype=dtype)
                v = pool[rng.integers(0, len(pool), (nz, ny, nx))]
            keys = bf.vertex_keys(v)
            flat = np.ascontiguousarray(v).reshape(-1)
            out = (ctypes.c_int64 * 17)()
            for vid in range(flat.size):
                h.harness_load_star(tables, code, flat.ctypes.data, nx, ny, nz, vid, out)
                L, rank, edge, _, _ = _star_cells(star, shape, vid, keys)
                present = 0
                x, y, z = vid % nx, (vid // nx) % ny, vid // (nx * ny)
                for n, (dx, dy, dz) in enumerate(offs):
                    if 0 <= x + dx < nx and 0 <= y + dy < ny and 0 <= z + dz < nz:
                        present |= 1 << n
                assert out[0] == present and out[1] == L, vid
                assert [out[3 + n] for n in range(14) if L >> n & 1] == \
                    [rank[n] for n in range(14) if L >> n & 1]
                lowest = [n for n in range(14) if L >> n & 1 and rank[n] == 0]
                assert out[2] == (lowest[0] if lowest else 0xF)


def test_order_keys_and_nan(star):
    """Key<T>::of orders like the numbers (-0.0 = +0.0, infinities at the
    ends) and Key<T>::nan finds every NaN, in float32 and float64."""
    h = _harness_extra(star)
    rng = np.random.default_rng(12)
    for dt, key, isnan, ubits in ((np.float32, h.harness_key_f32, h.harness_nan_f32, np.uint32),
                                  (np.float64, h.harness_key_f64, h.harness_nan_f64, np.uint64)):
        special = np.array([0.0, -0.0, np.inf, -np.inf, np.finfo(dt).max, -np.finfo(dt).max,
                            np.finfo(dt).tiny, -np.finfo(dt).tiny, np.finfo(dt).smallest_subnormal,
                            -np.finfo(dt).smallest_subnormal, 1.0, -1.0], dtype=dt)
        vals = np.concatenate([special, (rng.standard_normal(400) * 1e3).astype(dt),
                               rng.standard_normal(100).astype(dt) * np.finfo(dt).tiny])
        ks = [key(float(x)) for x in vals]
        for i in range(len(vals)):
            for j in range(0, len(vals), 7):
                a, b = vals[i], vals[j]
                assert (ks[i] < ks[j]) == (a < b) and (ks[i] == ks[j]) == (a == b), (a, b)
        nan_bits = [0x7FC00000, 0xFFC00000, 0x7F800001, 0xFFFFFFFF] if dt == np.float32 else \
            [0x7FF8000000000000, 0xFFF8000000000000, 0x7FF0000000000001, 0xFFFFFFFFFFFFFFFF]
        for b in nan_bits:
            x = np.array([b], dtype=ubits).view(dt)[0]
            assert isnan(float(x))
        assert not any(isnan(float(x)) for x in vals)
