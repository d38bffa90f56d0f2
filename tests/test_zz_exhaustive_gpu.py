"""Every vertex order of the 2x2x2 grid (8! = 40320 fields) through the CUDA
path, bit-exact against the oracle: the exhaustive property case of the
pairing on the smallest grid that holds all six tetrahedra of a cube."""
import itertools

import numpy as np
import pytest

import oracle
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


def test_every_vertex_order_of_a_cube(dms):
    with dms.Grid((2, 2, 2), np.float32) as g:
        for perm in itertools.permutations(range(8)):
            v = np.array(perm, dtype=np.float32).reshape(2, 2, 2)
            g.compute(v)
            diag = {d: g.fetch(d) for d in range(3)}
            compare(v, diag, oracle.pairsimplices(v))
