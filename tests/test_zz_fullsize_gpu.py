"""Parity at the full benchmark sizes, in the configuration bench.py times.

- Against the standard reduction itself: the oracle's fast mode was run on
  the full-size fields by tests/golden/make_oracle_digest.py, which stored,
  per dimension, the pair counts and the SHA-256 of the canonical pair list
  (and the SHA-256 of the field it ran on).  The GPU's pairs, put in the
  same canonical form, must hash the same: every pair of D0, D1 and D2 by
  simplex id and maximum vertex.
- Independently of those digests: D0 and D2 simplex for simplex against the
  union-find special cases, and D1 through the Euler characteristic of every
  sub-level set (chi(K_i) = #D0 alive - #D1 alive + #D2 alive at each vertex
  level i), which holds at any size."""
import json
import os

import numpy as np
import pytest

import oracle
import synthfields as sf
from tests.gpu_helpers import check_bits

pytestmark = pytest.mark.gpu


def _chi_by_level(v):
    """chi(K_i) for each vertex level i: each simplex counts (-1)^dim at the
    level of its maximum vertex (vectorised over the simplex types)."""
    nz, ny, nx = v.shape
    flat = v.reshape(-1)
    key = flat.astype(np.float64) if flat.dtype != np.float64 else flat
    order = np.lexsort((np.arange(flat.size), key))
    rank = np.empty(flat.size, np.int64)
    rank[order] = np.arange(flat.size)
    rank3 = rank.reshape(nz, ny, nx)
    delta = np.zeros(flat.size, np.int64)
    np.add.at(delta, rank, 1)
    tri = [(3, 1), (3, 2), (5, 1), (5, 4), (6, 2), (6, 4), (7, 1), (7, 2), (7, 3), (7, 4),
           (7, 5), (7, 6)]
    tet = [(1, 3), (1, 5), (2, 3), (2, 6), (4, 5), (4, 6)]

    def shifted(o, ext):
        dx, dy, dz = o & 1, (o >> 1) & 1, (o >> 2) & 1
        ex, ey, ez = ext & 1, (ext >> 1) & 1, (ext >> 2) & 1
        return rank3[dz:nz - ez + dz, dy:ny - ey + dy, dx:nx - ex + dx]

    for dim, chains in ((1, [(o,) for o in range(1, 8)]), (2, [(a, b) for b, a in tri]),
                        (3, [(a, b, 7) for a, b in tet])):
        for ch in chains:
            ext = max(ch)
            m = shifted(0, ext)
            for o in ch:
                m = np.maximum(m, shifted(o, ext))
            np.add.at(delta, m.reshape(-1), (-1) ** dim)
    return np.cumsum(delta), rank


def _gpu(values):
    import torch
    import paper_2206_13932_gb300 as dms
    nz, ny, nx = values.shape
    t = torch.from_numpy(values).cuda()
    with dms.Grid((nx, ny, nz), values.dtype) as g:
        g.compute(t)
        return {d: g.fetch(d) for d in range(3)}


def _check_full(v):
    diag = _gpu(v)
    check_bits(v, diag)
    d0 = {(int(p["birth_simplex"]), int(p["death_simplex"])) for p in diag[0]}
    k0 = {(int(r[1]), int(r[2])) for r in oracle.kruskal_d0(v)}
    assert d0 == k0
    d2 = {(int(p["birth_simplex"]), int(p["death_simplex"])) for p in diag[2]}
    k2 = {(int(r[1]), int(r[2])) for r in oracle.kruskal_d2(v)}
    assert d2 == k2
    chi, rank = _chi_by_level(v)
    alive = np.zeros(v.size + 1, np.int64)
    for d in range(3):
        p = diag[d]
        b = rank[p["birth_vertex"]]
        e = np.where(p["essential"] == 1, v.size, rank[np.maximum(p["death_vertex"], 0)])
        np.add.at(alive, b, (-1) ** d)
        np.add.at(alive, e, -((-1) ** d))
    assert np.array_equal(np.cumsum(alive)[: v.size], chi)


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2206_13932_gb300 as dms
    dms.build()


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _digest_check(name):
    from tests.golden.make_oracle_digest import canonical
    with open(os.path.join(GOLDEN, f"{name}_oracle.json")) as f:
        want = json.load(f)
    v = sf.config_field(name)               # on the CPU, as the digest was made
    assert sf.sha256(v) == want["field_sha256"], "the field differs from the oracle's input"
    diag = _gpu(v)
    check_bits(v, diag)
    rows = []
    for d in range(3):
        p = diag[d]
        rows.append(np.stack([p["dim"].astype(np.int64), p["birth_simplex"], p["death_simplex"],
                              p["birth_vertex"], p["death_vertex"],
                              p["essential"].astype(np.int64)], axis=1))
    got = canonical(np.concatenate(rows).astype(np.int64))
    for d in ("0", "1", "2"):
        assert got[d]["finite"] == want["dims"][d]["finite"], d
        assert got[d]["infinite"] == want["dims"][d]["infinite"], d
        assert got[d]["sha256"] == want["dims"][d]["sha256"], d


def test_noise256_f32_against_the_standard_reduction(gpu):
    """256^3 float32 white noise, seed 2: every pair equals the oracle's."""
    _digest_check("noise256_f32")


def test_mixture512_u16_against_the_standard_reduction(gpu):
    """The 512^3 uint16 recipe (64 Gaussians + 5 % noise, quantised: heavy
    ties), seed 3, at full size, in the configuration bench.py times: every
    pair equals the oracle's.  bench.py generates the field with torch on the
    GPU: it must be the same field, byte for byte."""
    _digest_check("mixture512_u16")
    import bench
    assert sf.sha256(bench.workload_field()) == sf.sha256(sf.config_field("mixture512_u16"))


def test_noise256_f32_full(gpu):
    """256^3 float32 white noise, seed 2 (57 % of vertices PL-critical)."""
    _check_full(sf.config_field("noise256_f32"))


def test_mixture_u16_quarter(gpu):
    """The 512^3 uint16 recipe at 256^3 (same blobs, noise and quantisation)."""
    _check_full(sf.config_field("mixture512_u16", shape_xyz=(256, 256, 256), device="cuda"))
