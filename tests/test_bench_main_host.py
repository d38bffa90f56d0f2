"""The bench's own arm run end to end on the host with fake device calls (no
GPU): every key of the one-line JSON contract is present and consistent,
the serving section runs through the server with a fake backend, and a
failure there is reported in its key instead of losing the line.  The
device numbers are made up by the fakes; only the bench's logic is checked.
"""
import contextlib
import io
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

torch = pytest.importorskip("torch")


class _FakeEvent:
    def __init__(self, enable_timing=False):
        pass

    def record(self, stream=None):
        pass

    def elapsed_time(self, other):
        return 12.5


class _FakeGrid:
    KERNELS = ("classify", "compact", "sort", "process_lower_stars", "emit", "d0_arcs",
               "d0_rounds", "d2_arcs", "d2_rounds", "d1_trace", "d1_reduce", "output")

    def __init__(self, shape_xyz, dtype):
        self.shape_xyz, self.dtype = tuple(shape_xyz), np.dtype(dtype)

    def compute(self, values, stream=None):
        return self

    def kernel_ms(self):
        return {k: (4.0 if k == "d1_reduce" else 1.0) for k in self.KERNELS}

    def stage_ms(self):
        return {k: 1.0 for k in ("gradient", "sort", "d0", "d2", "d1", "output", "total", "h2d")}

    def stats(self):
        return {"launches": 50, "d1_bytes_read": 10 ** 8, "d1_bytes_written": 5 * 10 ** 7,
                "c0": 10, "c1": 20, "c2": 30, "c3": 40, "d1_columns": 25, "d1_additions": 60}

    def work(self):
        return {"trace_toggles": 1000, "trace_expansions": 400, "d1_longest_chain": 8}

    def counts(self):
        return (3, 2, 1), (1, 0, 0, 0)

    def fetch(self, d, out=None):
        import paper_2206_13932_gb300 as dms
        p, e = self.counts()
        k = p[d] + e[d]
        res = np.zeros(k, dms.PAIR_DTYPE)
        if out is not None:
            assert out.dtype == dms.PAIR_DTYPE and len(out) >= k
            out[:k] = res
            return out[:k]
        return res

    def close(self):
        pass


@pytest.fixture
def fake_device(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    import paper_2206_13932_gb300 as dms
    from paper_2206_13932_gb300 import serve
    from tests.test_serve_host import _FakeBackend
    import synthfields as sf

    monkeypatch.setattr(torch.cuda, "set_device", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "Event", _FakeEvent)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a: object())
    monkeypatch.setattr(torch.Tensor, "cuda", lambda self, *a, **k: self)
    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self, *a, **k: self)
    real_empty = torch.empty
    monkeypatch.setattr(torch, "empty",
                        lambda *a, **k: real_empty(*a, **{x: y for x, y in k.items()
                                                          if x != "device"}))
    monkeypatch.setattr(dms, "build", lambda *a, **k: None)
    monkeypatch.setattr(dms, "Grid", _FakeGrid)
    monkeypatch.setattr(serve, "CudaBackend", _FakeBackend)
    monkeypatch.setattr(bench, "L2_BYTES", 4096)
    monkeypatch.setattr(bench, "ORACLE_SAMPLE", 8)
    monkeypatch.setitem(sf.CONFIGS, "mixture512_u16", ((16, 16, 16), np.uint16, "small"))
    small = [np.random.default_rng(i).random((4 + i % 3, 5, 6)).astype(np.float32)
             for i in range(12)]
    monkeypatch.setattr(sf, "serving_fields", lambda count, *a, **k: small)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    return bench


def _run(bench, argv):
    args = bench.argparse.Namespace(gpus=1, steps=2, warmup=3, impl="ours", no_serve=False)
    for k, v in argv.items():
        setattr(args, k, v)
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        bench.run_ours(args)
    lines = [ln for ln in out.getvalue().splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_one_line_with_every_contract_key(fake_device):
    d = _run(fake_device, {})
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e",
              "gpu_launches", "roofline", "cpu_baseline", "clocks"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 3
    assert d["ms_per_step"] == 12.5 and d["value"] == pytest.approx(16 ** 3 / 12.5e-3 / 1e6)
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["gpu_launches"] == 100
    assert set(d["e2e"]) == {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert d["e2e"]["h2d_bytes_per_step"] == 16 ** 3 * 2 and d["dtype"] == "u16"
    assert d["e2e"]["d2h_bytes_per_step"] == (4 + 2 + 1) * 56
    assert "512^3 uint16" in d["config"]["workload"]
    r = d["roofline"]                      # d1_reduce dominates the fake timings
    assert r == d["roofline_d1_reduce"] and r["bound"] == "hbm"
    assert r["achieved"] == pytest.approx(1.5e8 / 4e-3 / 1e9)      # merge bytes / time
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["longest_chain"] == 8 and r["us_per_chain_addition"] == pytest.approx(500.0)
    rg = d["roofline_gradient"]            # N*s_in + 8*|C| over classify+compact+PLS
    assert rg["algorithmic_bytes_per_launch"] == 16 ** 3 * 2 + 8 * 100
    assert rg["achieved"] == pytest.approx((16 ** 3 * 2 + 800) / 3e-3 / 1e9)
    assert rg["frac"] == pytest.approx(rg["achieved"] / rg["peak"])
    rc = d["roofline_classify"]
    assert rc["bound"] == "hbm" and rc["frac"] == pytest.approx(rc["achieved"] / rc["peak"])
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] > 0 and "sample" in cb
    assert cb["os_cpu_count"] == os.cpu_count() and "cpu_model" in cb and "host_ram_gib" in cb
    s = d["serving"]
    assert s["requests"] == 12 and s["saturated"]["one_at_a_time_rps"] > 0


def test_a_failing_serving_section_keeps_the_line(fake_device, monkeypatch):
    from paper_2206_13932_gb300 import serve

    def broken(*a, **k):
        raise RuntimeError("no server")
    monkeypatch.setattr(serve, "run_stream", broken)
    d = _run(fake_device, {})
    assert d["serving"] == {"error": "RuntimeError: no server"} and d["value"] > 0


def test_no_serve_skips_the_section(fake_device):
    assert _run(fake_device, {"no_serve": True})["serving"] is None


def test_dominant_pls_reports_the_issue_rate(fake_device, monkeypatch):
    """When ProcessLowerStars takes the most time, the headline roofline is
    its issue rate (an ALU-bound kernel), with the gradient stage's HBM figure
    beside it; a stale instruction count is reported as null."""
    def kms(self):
        return {k: (9.0 if k == "process_lower_stars" else 1.0) for k in self.KERNELS}
    import paper_2206_13932_gb300 as dms
    monkeypatch.setattr(dms.Grid, "kernel_ms", kms)
    d = _run(fake_device, {"no_serve": True})
    r = d["roofline"]
    assert r == d["roofline_pls"] and r["bound"] == "alu"
    assert r["peak"] == pytest.approx(152 * 4 * 2.07)
    stars = 16 ** 3          # 100 critical vertices of 4096, but a small grid: dense
    assert r["achieved"] == pytest.approx(
        fake_device.PLS_ISSUE["warp_inst_per_star"] * stars / 9e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert d["roofline_gradient"]["kernel"].startswith("gradient stage")
    monkeypatch.setitem(fake_device.PLS_ISSUE, "sources_sha256", "stale")
    d = _run(fake_device, {"no_serve": True})
    assert d["roofline"]["achieved"] is None and d["roofline"]["frac"] is None


def test_dominant_trace_reports_its_record_bytes(fake_device, monkeypatch):
    """When the D1 trace takes the most time, the headline roofline is its
    record reads (per toggle: record, flag, value, row word; per column: its
    entry, record and output slot) over its time, against HBM."""
    def kms(self):
        return {k: (9.0 if k == "d1_trace" else 1.0) for k in self.KERNELS}
    import paper_2206_13932_gb300 as dms
    monkeypatch.setattr(dms.Grid, "kernel_ms", kms)
    d = _run(fake_device, {"no_serve": True})
    r = d["roofline"]
    assert r == d["roofline_d1_trace"] and r["bound"] == "hbm"
    nbytes = 1000 * (48 + 1 + 2 + 8) + 25 * (9 + 48 + 13)
    assert r["algorithmic_bytes_per_launch"] == nbytes
    assert r["achieved"] == pytest.approx(nbytes / 9e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
