"""The bench's reference arm (the CPU oracle on bounded crops) prints one
JSON line with the contract's keys on rank 0, and nothing on other ranks."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       env=env, timeout=300, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-2000:]
    return [ln for ln in p.stdout.splitlines() if ln.startswith("{")]


def test_rank0_prints_one_line_with_the_contract_keys(monkeypatch):
    """In-process on a 24^3 stand-in of the workload (the 512^3 field takes a
    minute to generate on a CPU)."""
    import contextlib
    import io

    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    import synthfields as sf
    monkeypatch.setitem(sf.CONFIGS, "mixture512_u16", ((24, 24, 24), np.uint16, "small"))
    monkeypatch.setattr(bench, "REFERENCE_SAMPLE", 12)
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    args = bench.argparse.Namespace(gpus=1, steps=1, warmup=0, impl="reference", no_serve=True)
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        bench.run_reference(args)
    lines = [ln for ln in out.getvalue().splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["dtype"] == "u16"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["os_cpu_count"] == os.cpu_count()
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_other_ranks_exit_quietly():
    assert _run({"RANK": "1", "WORLD_SIZE": "2"}) == []


def test_traffic_hash_ignores_comments_only():
    """The stored DRAM traffic stays valid across comment edits, not code edits."""
    sys.path.insert(0, ROOT)
    import bench
    src = 'int f(int a) { // one\n  return a + 1; /* two\n */ }\nconst char *s = "a // b";\n'
    same = 'int f(int a) {\n  return a + 1; /* changed */ }\n// new line\nconst char *s = "a // b";\n'
    other = 'int f(int a) { // one\n  return a + 2; }\nconst char *s = "a // b";\n'
    assert bench._code_only(src) == bench._code_only(same)
    assert bench._code_only(src) != bench._code_only(other)
    assert '"a // b"' in bench._code_only(src)


def test_traffic_hash_covers_the_classification_code_only():
    """A change outside the classification code keeps the stored traffic; a
    change inside it, or a lost marker, drops it."""
    sys.path.insert(0, ROOT)
    import bench
    with open(os.path.join(ROOT, "paper_2206_13932_gb300", "csrc", "dms_pipeline.cu")) as f:
        src = f.read()
    base = bench._classify_code_of(src, "x")
    assert base is not None
    outside = src.replace("const int64_t nc = c.hst->total[0];",
                          "const int64_t nc = c.hst->total[0]; (void)0;")
    assert outside != src and bench._classify_code_of(outside, "x") == base
    inside = src.replace("struct ClsTiling {", "struct ClsTiling { int unused;", 1)
    assert inside != src and bench._classify_code_of(inside, "x") != base
    assert bench._classify_code_of(src, "y") != base
    lost = src.replace("stage 2: stable LSD radix sort", "stage 2")
    assert bench._classify_code_of(lost, "x") is None


def test_clock_summary_parses_the_sampled_lines():
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    c.lines = ["1965, 2070, 1100.5, Not Active, Not Active, Not Active, Active",
               "1980, 2070, 1180.2, Not Active, Not Active, Not Active, Not Active",
               "2010, 2070, 1200.0, Active, Not Active, Not Active, Not Active",
               "[N/A], 2070, 0, x, x, x, x", "garbage"]
    s = c.summary()
    assert s["sm_mhz"] == 1980 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert bench.ClockSampler(0).summary()["sm_mhz"] is None
