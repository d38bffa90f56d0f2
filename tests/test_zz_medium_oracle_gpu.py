"""Bit-exact parity at sizes where the D1 reduction meets its large-field
paths (long descending walls of smooth fields, the block expansion of the
lazy columns, heavy ties), against the sandwich oracle: ``oracle.sandwich``
runs the method's own steps on the CPU and is pinned to equal the standard
reduction (``tests/test_oracle_sandwich.py``); it finishes these fields in
tens of seconds where the full reduction needs minutes."""
import numpy as np
import pytest

import oracle
import synthfields as sf
from tests.gpu_helpers import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dms():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2206_13932_gb300 as m
    m.build()
    return m


def _gpu(dms, values, mode):
    import torch
    nz, ny, nx = values.shape
    with dms.Grid((nx, ny, nz), values.dtype, d1_mode=mode) as g:
        g.compute(torch.from_numpy(values.copy()).cuda())
        return {d: g.fetch(d) for d in range(3)}


@pytest.mark.parametrize("name", ["mixture112_f32", "recipe96_u16", "noise96_f32"])
def test_medium_fields_against_the_sandwich_oracle(dms, name):
    modes = (0, 1)
    if name == "mixture112_f32":        # smooth: few 2-saddles, long walls (lazy mode)
        v = sf.gaussian_mixture((112, 112, 112), 16, 1, noise=1e-3)
    elif name == "recipe96_u16":         # the 512^3 uint16 recipe at 96^3: heavy ties
        v = sf.quantize_u16(sf.gaussian_mixture((96, 96, 96), 64, 3, noise=0.05, dtype=None,
                                                noise_rel=True))
    else:                                # noise: many columns, long addition chains, the
        v = sf.white_noise((96, 96, 96), 2)     # asynchronous tail; every D1 mode
        modes = (0, 1, 2, 3)
    rows, _ = oracle.sandwich(v)
    for mode in modes:
        compare(v, _gpu(dms, v, mode), rows)
