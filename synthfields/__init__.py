"""Seeded synthetic scalar fields shaped like the paper's 3D volumes.

The paper benchmarks public volumes resampled to 192^3 plus an elevation and a
random field (Sec. 9.1).  Those volumes are not available here, so seeded
synthetic fields with the same structure stand in for them: smooth Gaussian
mixtures (few critical points, long integral lines), white noise (the paper's
"random" stress case, the largest diagrams) and quantised fields with heavy
ties.

This module holds no persistence arithmetic.  It is the one module that both
the oracle tests and the CUDA path consume; each field is generated once and
the same bytes are fed to both.  Arrays are indexed ``[z, y, x]`` so that x is
the fastest axis in memory (vertex id = x + nx*(y + ny*z)).
"""
from __future__ import annotations

import hashlib

import numpy as np

__all__ = ["gaussian_mixture", "white_noise", "quantize_u16", "ramp", "constant",
           "config_field", "sha256", "CONFIGS", "blob_params", "serving_shapes", "serving_fields",
           "serving_field", "poisson_arrivals"]


def blob_params(n_blobs: int, rng: np.random.Generator):
    """Centres U[0,1)^3, sigma U[0.05,0.2], amplitude random sign x U[0.5,1]."""
    centres = rng.random((n_blobs, 3))
    sigma = rng.uniform(0.05, 0.2, n_blobs)
    amp = rng.uniform(0.5, 1.0, n_blobs) * np.where(rng.random(n_blobs) < 0.5, -1.0, 1.0)
    return centres, sigma, amp


def _mixture_f64(shape_xyz, centres, sigma, amp, device=None):
    """Sum of isotropic Gaussians evaluated at p = (i/(nx-1), j/(ny-1), k/(nz-1)).

    Each Gaussian is separable, so it is formed as an outer product of three
    1D factors.  Runs on a torch device when one is given (same formula)."""
    nx, ny, nz = shape_xyz
    if device is not None:
        import torch
        dev = torch.device(device)
        ax = [torch.linspace(0.0, 1.0, n, dtype=torch.float64, device=dev) if n > 1 else
              torch.zeros(1, dtype=torch.float64, device=dev) for n in (nx, ny, nz)]
        g = torch.zeros((nz, ny, nx), dtype=torch.float64, device=dev)
        for c, s, a in zip(centres, sigma, amp):
            inv = 1.0 / (2.0 * float(s) * float(s))
            fx = torch.exp(-(ax[0] - float(c[0])) ** 2 * inv)
            fy = torch.exp(-(ax[1] - float(c[1])) ** 2 * inv)
            fz = torch.exp(-(ax[2] - float(c[2])) ** 2 * inv) * float(a)
            g += fz[:, None, None] * fy[None, :, None] * fx[None, None, :]
        return g
    ax = [np.linspace(0.0, 1.0, n) if n > 1 else np.zeros(1) for n in (nx, ny, nz)]
    g = np.zeros((nz, ny, nx), np.float64)
    for c, s, a in zip(centres, sigma, amp):
        inv = 1.0 / (2.0 * s * s)
        fx = np.exp(-(ax[0] - c[0]) ** 2 * inv)
        fy = np.exp(-(ax[1] - c[1]) ** 2 * inv)
        fz = np.exp(-(ax[2] - c[2]) ** 2 * inv) * a
        g += fz[:, None, None] * fy[None, :, None] * fx[None, None, :]
    return g


def gaussian_mixture(shape_xyz, n_blobs: int, seed: int, noise: float = 0.0,
                     dtype=np.float32, noise_rel: bool = False, device=None):
    """Gaussian mixture + uniform noise U(-noise, noise), generated in float64.

    ``noise_rel``: the noise half-width is ``noise * (max g - min g)``.
    With ``device`` set, the mixture is evaluated with torch on that device
    and returned as a numpy array (large grids)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    centres, sigma, amp = blob_params(n_blobs, rng)
    g = _mixture_f64(shape_xyz, centres, sigma, amp, device)
    if device is not None:
        g = g.cpu().numpy()
    if noise > 0:
        width = noise * (float(g.max()) - float(g.min())) if noise_rel else noise
        g = g + rng.uniform(-width, width, g.shape)
    return g.astype(dtype) if dtype is not None else g


def quantize_u16(g: np.ndarray) -> np.ndarray:
    """round(65535 * (g - min) / (max - min)) as uint16 (heavy ties)."""
    lo, hi = float(g.min()), float(g.max())
    scale = 65535.0 / (hi - lo) if hi > lo else 0.0
    return np.rint((g - lo) * scale).astype(np.uint16)


def white_noise(shape_xyz, seed: int, dtype=np.float32):
    """iid U[0,1) (the paper's "random" stress case)."""
    nx, ny, nz = shape_xyz
    rng = np.random.Generator(np.random.PCG64(seed))
    if np.dtype(dtype) == np.uint16:
        return rng.integers(0, 65536, (nz, ny, nx), dtype=np.uint16)
    return rng.random((nz, ny, nx), dtype=np.float64).astype(dtype)


def ramp(shape_xyz, dtype=np.float32):
    """f = x + y + z (the elevation case: a single infinite bar)."""
    nx, ny, nz = shape_xyz
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return (x + y + z).astype(dtype)


def constant(shape_xyz, dtype=np.float32, value=1.0):
    nx, ny, nz = shape_xyz
    return np.full((nz, ny, nx), value, dtype=dtype)


def sha256(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


# The named workloads.  (shape_xyz, dtype, recipe)
CONFIGS = {
    "mixture32_f32": ((32, 32, 32), np.float32,
                      "16 Gaussians + U(-1e-3, 1e-3) noise, seed 1"),
    "noise256_f32": ((256, 256, 256), np.float32, "iid U[0,1), seed 2"),
    "mixture512_u16": ((512, 512, 512), np.uint16,
                       "64 Gaussians + uniform noise of half-width 0.05*(max-min), "
                       "quantised to uint16, seed 3"),
}


def config_field(name: str, device=None, shape_xyz=None) -> np.ndarray:
    """The seeded field of a named workload (optionally at another shape)."""
    shape, dtype, _ = CONFIGS[name]
    shape = tuple(shape_xyz) if shape_xyz is not None else shape
    if name == "mixture32_f32":
        return gaussian_mixture(shape, 16, 1, noise=1e-3, dtype=np.float32, device=device)
    if name == "noise256_f32":
        return white_noise(shape, 2, np.float32)
    if name == "mixture512_u16":
        g = gaussian_mixture(shape, 64, 3, noise=0.05, noise_rel=True, dtype=None,
                             device=device)
        return quantize_u16(g)
    raise KeyError(name)


def serving_shapes(count: int, seed: int = 4000, lo: int = 16, hi: int = 128):
    """Per-axis sizes round(exp(U(ln lo, ln hi))), drawn independently."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [tuple(int(round(np.exp(rng.uniform(np.log(lo), np.log(hi))))) for _ in range(3))
            for _ in range(count)]


def serving_fields(count: int, seed0: int = 4000, lo: int = 16, hi: int = 128):
    """The serving workload: fields of log-uniform non-cubic shapes, each
    16 Gaussians + U(-1e-3, 1e-3) noise in float32, seeds seed0 + i."""
    shapes = serving_shapes(count, seed0, lo, hi)
    return [gaussian_mixture(sh, 16, seed0 + i, noise=1e-3, dtype=np.float32)
            for i, sh in enumerate(shapes)]


def serving_field(i: int, seed0: int = 4000, lo: int = 16, hi: int = 128):
    """Field i of :func:`serving_fields` alone (the same shape and bytes)."""
    shape = serving_shapes(i + 1, seed0, lo, hi)[i]
    return gaussian_mixture(shape, 16, seed0 + i, noise=1e-3, dtype=np.float32)


def poisson_arrivals(count: int, rate_per_s: float, seed: int = 4100):
    """Arrival times (seconds) of a Poisson process of the given rate."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate_per_s, count))
