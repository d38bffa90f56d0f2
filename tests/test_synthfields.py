"""The seeded input generators (shared by the CUDA path's tests and the
oracle's): deterministic per seed, the documented shapes, dtypes and value
ranges, the separable mixture equal to its direct sum, and the serving
workload's shape and arrival recipes."""
import numpy as np
import pytest

import synthfields as sf


def test_same_seed_same_bytes_other_seed_other_bytes():
    a, b = sf.white_noise((9, 8, 7), 2), sf.white_noise((9, 8, 7), 2)
    assert sf.sha256(a) == sf.sha256(b) and sf.sha256(a) != sf.sha256(sf.white_noise((9, 8, 7), 3))
    m1 = sf.gaussian_mixture((10, 9, 8), 4, 5, noise=1e-3)
    m2 = sf.gaussian_mixture((10, 9, 8), 4, 5, noise=1e-3)
    assert sf.sha256(m1) == sf.sha256(m2)


def test_shapes_dtypes_and_ranges():
    n = sf.white_noise((6, 5, 4), 1)
    assert n.shape == (4, 5, 6) and n.dtype == np.float32 and 0 <= n.min() and n.max() < 1
    u = sf.white_noise((6, 5, 4), 1, np.uint16)
    assert u.dtype == np.uint16
    q = sf.quantize_u16(np.linspace(-3.0, 5.0, 101))
    assert q.dtype == np.uint16 and q.min() == 0 and q.max() == 65535
    assert sf.quantize_u16(np.zeros(4)).tolist() == [0, 0, 0, 0]
    r = sf.ramp((4, 3, 2))
    assert r[1, 2, 3] == 6 and sf.constant((2, 2, 2), value=3.0).sum() == 24


def test_mixture_is_the_direct_sum_of_its_gaussians():
    shape = (7, 6, 5)
    rng = np.random.Generator(np.random.PCG64(9))
    centres, sigma, amp = sf.blob_params(3, rng)
    g = sf.gaussian_mixture(shape, 3, 9)
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.linspace(0, 1, nz), np.linspace(0, 1, ny), np.linspace(0, 1, nx),
                          indexing="ij")
    want = sum(a * np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (2 * s * s))
               for c, s, a in zip(centres, sigma, amp))
    assert np.allclose(g, want.astype(np.float32), rtol=1e-6, atol=1e-7)
    assert np.all((0.05 <= sigma) & (sigma <= 0.2)) and np.all(np.abs(amp) >= 0.5)


def test_named_workloads():
    assert set(sf.CONFIGS) == {"mixture32_f32", "noise256_f32", "mixture512_u16"}
    small = sf.config_field("mixture512_u16", shape_xyz=(8, 8, 8))
    assert small.dtype == np.uint16 and small.shape == (8, 8, 8)
    assert sf.config_field("mixture32_f32").shape == (32, 32, 32)
    with pytest.raises(KeyError):
        sf.config_field("nothing")


def test_serving_recipe():
    shapes = sf.serving_shapes(400)
    assert shapes == sf.serving_shapes(400)
    edges = np.array(shapes).ravel()
    assert edges.min() >= 16 and edges.max() <= 128
    # log-uniform: about half the edges below the geometric mean of the range
    assert abs(np.mean(edges < np.sqrt(16 * 128)) - 0.5) < 0.08
    t = sf.poisson_arrivals(2000, 100.0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0) and abs(gaps.mean() - 0.01) < 0.001
