"""Differentiable persistence diagrams (torch.autograd).

The value of a persistence pair is the value of the maximum vertices of its
two simplices (Sec. 2.4: persistence = f(max vertex of the death simplex) -
f(max vertex of the birth simplex)).  For a fixed pairing the births and
deaths are therefore entries of the field, and the gradient of any loss of
the diagram scatters onto those vertices.  The forward pass runs the CUDA
pipeline; the backward pass runs the scatter kernel behind
``dms_backward_pairs``.  The pairing is piecewise constant in the field;
where it changes (ties, crossings) the gradient is that of the current
pairing.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import PAIR_DTYPE, Grid, _check

_REC = PAIR_DTYPE.itemsize   # 56 bytes per pair


@dataclass
class Diagram:
    """Pairs of one dimension.  ``birth``/``death`` are differentiable."""
    birth: torch.Tensor
    death: torch.Tensor
    essential: torch.Tensor          # bool
    birth_vertex: torch.Tensor       # int64
    death_vertex: torch.Tensor       # int64 (-1 for infinite classes)
    birth_simplex: torch.Tensor
    death_simplex: torch.Tensor


def _fetch_device(grid: Grid, dim: int, count: int) -> torch.Tensor:
    buf = torch.empty(max(count, 1) * _REC, dtype=torch.uint8, device="cuda")
    if count:
        grid.fetch_device(dim, buf.data_ptr(), count)
    return buf[: count * _REC].view(count, _REC)


def _bits_to_values(bits: torch.Tensor, dtype: torch.dtype) -> torch.Tensor:
    if dtype == torch.float32:
        return bits.to(torch.int32).view(torch.float32)
    if dtype == torch.float64:
        return bits.view(torch.float64)
    return bits.to(torch.float32)    # uint16 values (not differentiable fields)


class _DiagramFn(torch.autograd.Function):
    """Connects the births and deaths (read off the pair records) to the
    field; backward scatters their gradients with dms_backward_pairs."""

    @staticmethod
    def forward(ctx, values, grid, counts, result_id, *bd):
        ctx.grid = grid
        ctx.result_id = result_id
        ctx.shape = values.shape
        ctx.dtype = values.dtype
        ctx.counts = counts
        return tuple(t.clone() for t in bd)

    @staticmethod
    def backward(ctx, *grads):
        grid = ctx.grid
        n = int(np.prod(ctx.shape))
        gfield = torch.zeros(n, dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        for d in range(3):
            gb, gd = grads[2 * d], grads[2 * d + 1]
            if ctx.counts[d] == 0 or (gb is None and gd is None):
                continue
            gb = gb.to(torch.float64).contiguous() if gb is not None else None
            gd = gd.to(torch.float64).contiguous() if gd is not None else None
            _check(grid._lib.dms_backward_pairs(
                grid._h, d, ctx.result_id, ctypes.c_void_p(gb.data_ptr() if gb is not None else 0),
                ctypes.c_void_p(gd.data_ptr() if gd is not None else 0),
                ctypes.c_void_p(gfield.data_ptr()), ctypes.c_void_p(int(stream))),
                "dms_backward_pairs")
        return (gfield.to(ctx.dtype).view(ctx.shape), None, None, None) + (None,) * len(grads)


def persistence_diagram(values: torch.Tensor, grid: Grid | None = None) -> list:
    """D0, D1, D2 of a CUDA field indexed [z, y, x] (float32 or float64), with
    births and deaths differentiable with respect to ``values``.  ``grid`` (a
    :class:`Grid` of the field's shape and dtype) may be reused across calls;
    it must stay alive until the backward pass has run, and the backward pass
    refuses (DMS_ERR_STATE) once the grid has computed another field since,
    because its pairs are no longer the ones these diagrams hold.  With a :class:`Batch`
    as ``grid``, ``values`` holds its fields packed one after another and the
    diagrams hold every field's pairs, grouped by field (``grid.offsets(d)``
    gives the ranges); the gradient comes back in the packed layout."""
    if not values.is_cuda:
        raise ValueError("values must be a CUDA tensor")
    values = values.contiguous()
    if grid is None:
        nz, ny, nx = values.shape
        grid = Grid((nx, ny, nz), np.dtype(str(values.dtype).replace("torch.", "")))
    grid.compute(values.detach())
    pairs, ess = grid.counts()
    counts = tuple(grid.list_rows(d) for d in range(3))
    bd, meta = [], []
    for d in range(3):
        n = counts[d]
        rec = _fetch_device(grid, d, n)
        i64 = rec[:, :48].contiguous().view(torch.int64).view(n, 6)
        bd += [_bits_to_values(i64[:, 4].contiguous(), values.dtype),
               _bits_to_values(i64[:, 5].contiguous(), values.dtype)]
        meta.append((rec[:, 49].to(torch.bool), i64[:, 2].clone(), i64[:, 3].clone(),
                     i64[:, 0].clone(), i64[:, 1].clone()))
    outs = _DiagramFn.apply(values, grid, counts, grid.result_id(), *bd)
    return [Diagram(outs[2 * d], outs[2 * d + 1], *meta[d]) for d in range(3)]


def persistence_loss(diagrams: list, threshold: float = 0.01, dims=(0, 2)) -> torch.Tensor:
    """Sum over the finite pairs of the given dimensions with persistence
    above ``threshold`` of persistence squared."""
    total = None
    for d in dims:
        dg = diagrams[d]
        p = dg.death - dg.birth
        keep = (~dg.essential) & (p > threshold)
        term = (p[keep] ** 2).sum()
        total = term if total is None else total + term
    return total
