"""The tunables change the speed of a compute, never its pairs; the autotuner
returns valid values and leaves the handle set to them."""
import numpy as np
import pytest

import synthfields as sf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dms():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2206_13932_gb300 as m
    m.build()
    return m


def test_every_candidate_gives_the_same_pairs(dms):
    from paper_2206_13932_gb300 import autotune as at
    for v in (sf.white_noise((48, 40, 36), 8), sf.gaussian_mixture((48, 48, 48), 10, 9,
                                                                   noise=1e-3)):
        with dms.Grid((v.shape[2], v.shape[1], v.shape[0]), v.dtype) as g:
            g.compute(v)
            want = {d: g.fetch(d).tobytes() for d in range(3)}
            for k, name in enumerate(at.TUNABLES):
                for cand in at.CANDIDATES[name] + ((8, 1024) if "heap" in name else ()):
                    vals = tuple(cand if i == k else x for i, x in enumerate(at.DEFAULT))
                    if not at.valid(vals):
                        continue
                    at.set_tuning(g, vals)
                    g.compute(v)
                    for d in range(3):
                        assert g.fetch(d).tobytes() == want[d], (name, cand, d)
            at.set_tuning(g, at.DEFAULT)


def test_out_of_range_values_are_refused(dms):
    from paper_2206_13932_gb300 import autotune as at
    with dms.Grid((8, 8, 8), np.float32) as g:
        for k, bad in ((0, 48), (0, 1024), (1, 16), (1, 512), (2, 100), (3, 4), (5, 2000), (6, 0), (7, 2),
                       (8, 3), (4, -2), (9, 2)):
            vals = tuple(bad if i == k else x for i, x in enumerate(at.DEFAULT))
            with pytest.raises(dms.DmsError):
                at.set_tuning(g, vals)
        assert at.get_tuning(g) == at.DEFAULT


def test_tune_returns_a_valid_setting(dms, tmp_path):
    from paper_2206_13932_gb300 import autotune as at
    v = sf.white_noise((64, 64, 64), 12)
    with dms.Grid((64, 64, 64), np.float32) as g:
        best, info = at.tune(g, v, repeats=2)
        assert at.valid(best) and at.get_tuning(g) == best
        assert info["best_ms"] <= info["start_ms"]
        path = str(tmp_path / "tuning.json")
        key = at.cache_key(np.float32, 64 ** 3)
        at.save(path, key, best)
        assert at.load(path, key) == best
