"""The library's lower-star code, run on the host, against the oracle.

``tests/host/pls_host.cc`` compiles ``csrc/dms_common.cuh`` (the code the
kernels run) for the host, with the star tables the library builds
(``dms_star_tables``); ``tests/pls_checks.py`` drives it.  No GPU is
involved: this pins the logic of the gradient kernels, and the GPU parity
tests pin their device build.

- ProcessLowerStars: for every lower star of small random fields (with and
  without ties, boundary vertices included) and for every lower-link mask of
  an interior vertex, the critical cells and pairs equal the oracle's gradient
  (Alg. 2, ``oracle/sandwich.c``) restricted to that star, simplex for simplex.
- The classification's table of PL-regular masks (``dms_regular_table``)
  marks exactly the masks whose lower star has no critical cell (Sec. 2.6).
- The star view (``load_star``) and the order keys (``Key<T>``) follow the
  order by (value, vertex id) of Sec. 2.1, with ties, signed zeros and
  infinities; every NaN is found.
- Plausible mistakes planted in a copy of the header are caught.
"""
import ctypes
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

from tests import pls_checks as pc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _have_tools():
    return shutil.which("g++") is not None and os.path.isdir(pc.CUDA_INCLUDE)


@pytest.fixture(scope="module")
def hv(tmp_path_factory):
    if not _have_tools():
        pytest.skip("needs g++ and the CUDA headers")
    out = str(tmp_path_factory.mktemp("plshost") / "libplshost.so")
    return pc.Harness(pc.build_harness(pc.CSRC, out))


@pytest.mark.parametrize("kind", ["float", "ties", "perm", "signed"])
def test_every_lower_star_of_random_fields(hv, kind):
    rng = np.random.default_rng({"float": 1, "ties": 2, "perm": 3, "signed": 4}[kind])
    for shape in [(3, 3, 3), (4, 3, 3), (3, 4, 2), (2, 2, 2), (5, 3, 1)]:
        for _ in range(6):
            pc.check_field(hv, pc.random_field(rng, shape, kind))


def test_every_lower_link_mask_of_an_interior_vertex(hv):
    """All 2^14 lower masks of the centre of a 3x3x3 grid, each with random
    values (so random ranks) on its lower and upper neighbours; the regular
    table marks exactly the masks without a critical cell."""
    import paper_2206_13932_gb300 as dms
    lib = dms.load()
    lib.dms_regular_table.restype = ctypes.c_int64
    lib.dms_regular_table.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    words = lib.dms_regular_table(None, 0)
    assert words == (1 << 14) // 32
    table = (ctypes.c_uint32 * words)()
    assert lib.dms_regular_table(table, words) == words
    rng = np.random.default_rng(7)
    centre = 13
    link_ids = [(1 + dx) + 3 * ((1 + dy) + 3 * (1 + dz)) for dx, dy, dz in hv.offs]
    regular = 0
    for m in range(1 << 14):
        v = rng.random(27) + 2.0                     # everything above the centre
        v[centre] = 1.5
        for n in range(14):
            if m >> n & 1:
                v[link_ids[n]] = rng.random()        # below the centre
        crit = pc.check_field(hv, v.reshape(3, 3, 3), vertices=[centre])
        is_regular = not crit.get(centre)
        assert bool(table[m >> 5] >> (m & 31) & 1) == is_regular, m
        regular += is_regular
    assert 0 < regular < 1 << 14


@pytest.mark.parametrize("dtype", [np.uint16, np.float32, np.float64])
def test_star_view_follows_the_vertex_order(hv, dtype):
    rng = np.random.default_rng(11)
    for shape in [(3, 3, 3), (5, 4, 3), (4, 1, 6), (1, 1, 5)]:
        for _ in range(4):
            pc.check_star_view(hv, pc.random_field(rng, shape, "ties").astype(dtype))
            if dtype != np.uint16:
                pc.check_star_view(hv, pc.random_field(rng, shape, "signed").astype(dtype))


def test_order_keys_and_nan(hv):
    """Key<T>::of orders like the numbers (-0.0 = +0.0, infinities at the
    ends) and Key<T>::nan finds every NaN, in float32 and float64."""
    h = hv.h
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


# (name, exact text of dms_common.cuh, replacement); the text occurs once
MUTANTS = [
    ("the vertex paired with its highest edge",
     "const int n0 = (int)(lrw & 15);", "const int n0 = (int)((lrw >> (4 * (p - 1))) & 15);"),
    ("triangles of one highest rank in the wrong order",
     "for (int lo = 0; lo < hi; lo++) {", "for (int lo = hi - 1; lo >= 0; lo--) {"),
    ("tets of one triangle in the wrong order",
     "for (int t = 0; t < lo; t++) {", "for (int t = lo - 1; t >= 0; t--) {"),
    ("PQzero edges taken out of order",
     "const int re = zr ? __ffs(zr) - 1 : kLinks;",
     "const int re = zr ? __ffs((zr & (zr - 1)) ? (zr & (zr - 1)) : zr) - 1 : kLinks;"),
    ("no edge waits in PQzero", "    zr = ((1u << p) - 1) & ~1u;", "    zr = 0;"),
    ("ties decided against the vertex id",
     "bool lo = kn[n] < kv || (kn[n] == kv && n >= 7);",
     "bool lo = kn[n] < kv || (kn[n] == kv && n < 7);"),
    ("ranks of tied neighbours reversed",
     "pk[n] = ((P)kn[n] << 4) | (P)(n < 7 ? 7 + n : 13 - n);",
     "pk[n] = ((P)kn[n] << 4) | (P)(n < 7 ? 6 - n : n);"),
    ("ranks of tied neighbours reversed (float64)",
     "(kn[m] < kn[n] || (kn[m] == kn[n] && g.dlin[m] < g.dlin[n]))",
     "(kn[m] < kn[n] || (kn[m] == kn[n] && g.dlin[m] > g.dlin[n]))"),
    ("negative floats not flipped",
     "        return (u & 0x80000000u) ? ~u : (u | 0x80000000u);",
     "        return u | 0x80000000u;"),
    ("a tet face left out of its unclassified faces",
     "((1ull << S.tet_f[h][0]) | (1ull << S.tet_f[h][1]) | (1ull << S.tet_f[h][2])) & ~cT",
     "((1ull << S.tet_f[h][0]) | (1ull << S.tet_f[h][1])) & ~cT"),
]


def _run_checks(include_dir):
    return subprocess.run([sys.executable, "-m", "tests.pls_checks", str(include_dir)],
                          cwd=ROOT, capture_output=True, text=True, timeout=600)


def test_unmodified_header_passes_the_compact_checks(tmp_path):
    if not _have_tools():
        pytest.skip("needs g++ and the CUDA headers")
    shutil.copy(os.path.join(pc.CSRC, "dms_common.cuh"), tmp_path)
    r = _run_checks(tmp_path)
    assert r.returncode == 0, r.stdout + r.stderr


@pytest.mark.parametrize("name,text,repl", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_in_the_header_is_caught(tmp_path, name, text, repl):
    if not _have_tools():
        pytest.skip("needs g++ and the CUDA headers")
    src = open(os.path.join(pc.CSRC, "dms_common.cuh")).read()
    assert src.count(text) == 1, "the planted text must occur once"
    with open(os.path.join(tmp_path, "dms_common.cuh"), "w") as f:
        f.write(src.replace(text, repl))
    r = _run_checks(tmp_path)
    assert r.returncode != 0, f"not caught: {name}"
