"""Host side of the autotuner (no GPU): candidate validity, cache keys and
the JSON cache."""
import numpy as np

from paper_2206_13932_gb300 import autotune as at


def test_defaults_and_candidates_are_valid_settings():
    assert len(at.DEFAULT) == len(at.TUNABLES)
    assert at.valid(at.DEFAULT)
    for k, name in enumerate(at.TUNABLES):
        assert at.DEFAULT[k] in at.CANDIDATES[name]
        for cand in at.CANDIDATES[name]:
            vals = tuple(cand if i == k else x for i, x in enumerate(at.DEFAULT))
            assert at.valid(vals), (name, cand)


def test_trace_threads_must_be_whole_blocks():
    vals = list(at.DEFAULT)
    vals[at.TUNABLES.index("trace_block")] = 256
    vals[at.TUNABLES.index("trace_per_sm")] = 128
    assert not at.valid(vals)


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    k1 = at.cache_key(np.float32, 256 ** 3, 0)
    k2 = at.cache_key(np.uint16, 512 ** 3, 3)
    assert k1 != k2 and at.cache_key(np.float32, 256 ** 3 + 5, 0) == k1
    assert at.load(path, k1) is None
    at.save(path, k1, at.DEFAULT)
    at.save(path, k2, tuple(reversed(at.DEFAULT)))
    assert at.load(path, k1) == at.DEFAULT
    assert at.load(path, k2) == tuple(reversed(at.DEFAULT))


def test_valid_mirrors_the_ranges_the_library_accepts():
    """The refusals of dms_set_tuning (checked on a GPU in
    test_autotune_gpu.py) are refused here already."""
    for k, bad in ((0, 48), (0, 1024), (1, 16), (1, 512), (2, 100), (3, 4), (5, 2000), (6, 0),
                   (7, 2), (8, 3), (2, 16384), (4, -2), (9, 2)):
        vals = tuple(bad if i == k else x for i, x in enumerate(at.DEFAULT))
        assert not at.valid(vals), (at.TUNABLES[k], bad)
    assert not at.valid(at.DEFAULT[:-1])


class _FakeLib:
    """dms_get_tuning / dms_set_tuning over a plain list, refusing what
    autotune.valid refuses (as the library does)."""

    def __init__(self):
        self.values = list(at.DEFAULT)

    def dms_get_tuning(self, h, v, count):
        for i in range(count):
            v[i] = self.values[i]
        return 0

    def dms_set_tuning(self, h, v, count):
        vals = [int(v[i]) for i in range(count)]
        if not at.valid(vals):
            return 1
        self.values = vals
        return 0


class _FakeGrid:
    """A device time that is a separable function of the tunables, smallest at
    ``best``."""

    def __init__(self, best):
        self._lib, self._h, self.best = _FakeLib(), None, best

    def compute(self, field):
        pass

    def stage_ms(self):
        cost = 10.0
        for k, name in enumerate(at.TUNABLES):
            cands = at.CANDIDATES[name]
            cost += abs(cands.index(self._lib.values[k]) - cands.index(self.best[k]))
        return {"total": cost}


def test_tune_finds_the_best_of_a_separable_cost_and_leaves_it_set():
    best = tuple(c[-1] for c in at.CANDIDATES.values())
    assert at.valid(best)
    g = _FakeGrid(best)
    vals, info = at.tune(g, None, repeats=1)
    assert vals == best and tuple(g._lib.values) == best
    assert info["best_ms"] == 10.0 and info["start_ms"] > info["best_ms"]
    assert all(at.valid(v) for v, _ in info["trials"])


def test_tune_keeps_the_defaults_when_nothing_gains_enough():
    g = _FakeGrid(at.DEFAULT)
    vals, info = at.tune(g, None, repeats=1, min_gain=0.5)
    assert vals == at.DEFAULT and info["best_ms"] == info["start_ms"]
