"""Benchmark of the full D0/D1/D2 pipeline on one GPU (or N independent
replicas under torchrun), printing one JSON line.

Workload: the 512^3 uint16 field (64 Gaussians + uniform noise of half-width
5 % of the range, quantised: heavy ties broken by vertex id, seed 3), one
field per step -- the largest single-GPU configuration.  A step is one pass
of the whole pipeline (gradient, critical simplices, D0, D2, D1, output) over
that field.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the standard reduction of Alg. 1) on
bounded sub-volumes of the same field, on this machine's host cores.

Rooflines in the line: ``roofline`` for the kernel family that takes the most
device time, ``roofline_d1_trace`` for the D1 boundary trace against the
record bytes its walks read, ``roofline_d1_reduce`` for the D1 reduction
(its merge bytes, and its longest chain of additions with the time per
link), ``roofline_pls`` for ProcessLowerStars against the issue rate,
``roofline_gradient`` for the gradient stage (classification, compaction and
ProcessLowerStars) against its algorithmic bytes N*s_in + 8*|C| (every value
read once, every critical simplex written once), and ``roofline_classify``
for the per-vertex stencil alone.  ``e2e_split_ms`` splits the end-to-end
step into the compute call, its host-to-device copy and the fetches.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthfields as sf  # noqa: E402

WORKLOAD = "mixture512_u16"
WORKLOAD_TEXT = ("512^3 uint16: 64 Gaussians + uniform noise of half-width 0.05*(max-min), "
                 "quantised to uint16 (heavy ties), seed 3 (one field per step)")
DTYPE_NAME = "u16"
SMS, SMSPS, SM_MAX_MHZ = 152, 4, 2070.0    # GB300: issue peak = SMs x schedulers x clock
METRIC = "full-diagram Mvertices/s"
UNIT = "Mvertices/s"
L2_BYTES = 129 * 2**20
ORACLE_SAMPLE = 96          # edge of the cube cropped for the oracle (cpu_baseline)
SERVE_REQUESTS = 1024       # requests of the serving workload replayed per run
SERVE_BATCH = 16            # most requests one batched pass takes
# DRAM bytes per launch of the classification stencil on this workload, from
# one ncu capture (profiles/classify_u16_512.md), valid only for the code it
# was taken on (sha256 of the code behind that kernel, comments excluded:
# _CLASSIFY_SPANS); otherwise reported as null.
CLASSIFY_TRAFFIC = {"sources_sha256": "549b412bd718737b55508d3b5f790f81571780dce33b77c61faf823f22740f0f",
                    "bytes_per_launch": 268509184 + 118023680}
# Warp instructions issued per star by ProcessLowerStars' two kernels
# (k_pls_keys + k_pls_run), from one ncu capture (profiles/pls_two_pass_noise192.md:
# 201 719 808 + 2 692 079 773 instructions for 7 077 888 stars of 192^3 noise,
# 57 % of them PL-critical, like this workload), valid only for the code it
# was taken on (_PLS_SPANS).  The radix sort between the two passes is not
# counted, so the achieved rate is a slight underestimate.
PLS_ISSUE = {"sources_sha256": "d18c3c097185b93f1690f54cbdf3f2eb4bc8fe34227170c46b7e11189ff847e0",
             "warp_inst_per_star": (201719808 + 2692079773) / 7077888, "simt_lanes": 14.9,
             "alu_pipe_pct_run": 67.9}


def _code_only(src: str) -> str:
    """C++ source without its comments, whitespace runs collapsed: editing a
    comment does not change what the compiler sees."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


# The code that decides the classification kernel's DRAM traffic, as
# (start, end) markers in dms_pipeline.cu: the star tables and utilities, the
# classification stage (its kernels), the tiling of its launch, and the launch
# itself.  dms_common.cuh counts whole.
_CLASSIFY_SPANS = (("// ------------------------------------------------------------ host tables",
                    "// ------------------------------------------------------------------ scan"),
                   ("// --------------------------------------------------- stage 1: classification",
                    "stage 2: stable LSD radix sort"),
                   ("struct ClsTiling", "struct Ctx"), ("k_classify2<T><<<", ");"))


# The code behind the instruction count of ProcessLowerStars in the bench:
# its two kernels (the counted ones; the radix sort between them is not
# counted); dms_common.cuh (star view, ProcessLowerStars) counts whole.
_PLS_SPANS = (("__global__ void __launch_bounds__(256)\n    k_pls_keys(",
               "// The critical cells of the lower star of each sorted"),)


def _code_of(pipeline_src: str, common_src: str, spans):
    """Comment-free text of the code behind a kernel (dms_common.cuh and the
    spans of dms_pipeline.cu between each pair of markers), or None when a
    marker is missing."""
    parts = [common_src]
    for a, b in spans:
        i = pipeline_src.find(a) if a else 0
        j = pipeline_src.find(b, i + len(a)) if i >= 0 else -1
        if i < 0 or j < 0:
            return None
        parts.append(pipeline_src[i:j + len(b)])
    return "\0".join(_code_only(p) for p in parts)


def _classify_code_of(pipeline_src: str, common_src: str):
    """Comment-free text of the code behind the classification kernel, or None
    when a marker is missing."""
    return _code_of(pipeline_src, common_src, _CLASSIFY_SPANS)


def _kernel_sources_sha256(spans=_CLASSIFY_SPANS):
    """Hash of the code (comments excluded) behind a kernel (by default the
    classification's): a stored ncu figure is reported only while it matches."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2206_13932_gb300", "csrc")
    with open(os.path.join(csrc, "dms_pipeline.cu")) as f:
        pipeline_src = f.read()
    with open(os.path.join(csrc, "dms_common.cuh")) as f:
        common_src = f.read()
    code = _code_of(pipeline_src, common_src, spans)
    return None if code is None else hashlib.sha256(code.encode()).hexdigest()


REFERENCE_SAMPLE = 64       # edge of the crop per reference-arm step


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.t:
                self.t.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def host_info():
    """The host the oracle runs on: CPU model, logical CPUs, RAM."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    ram = None
    try:
        with open("/proc/meminfo") as f:
            ram = round(int(f.readline().split()[1]) / 2**20, 1)
    except (OSError, ValueError, IndexError):
        pass
    import platform
    return {"cpu_model": model, "machine": platform.machine(), "os_cpu_count": os.cpu_count(),
            "host_ram_gib": ram}


def workload_field():
    """The bench field, generated with torch on the GPU when there is one (the
    Gaussians only; the same formula and seeds as on the CPU)."""
    dev = None
    try:
        import torch
        dev = "cuda" if torch.cuda.is_available() else None
    except ImportError:
        pass
    return sf.config_field(WORKLOAD, device=dev)


def _oracle_sample(field, edge):
    """Times the oracle -- the standard reduction of the lexicographic
    filtration in its fast mode (clearing, implicit apparent columns, a
    streamed filtration; the textbook mode's pairs) -- on an edge^3 corner
    crop of the field (CPU, one thread)."""
    import oracle
    oracle.build()
    crop = np.ascontiguousarray(field[:edge, :edge, :edge])
    t0 = time.perf_counter()
    rows = oracle.fastpairs(crop)
    dt = time.perf_counter() - t0
    return crop.size, dt, len(rows)


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return
    field = workload_field()
    for _ in range(args.warmup):
        _oracle_sample(field, 16)
    tot_v, tot_t = 0, 0.0
    for _ in range(args.steps):
        nv, dt, _ = _oracle_sample(field, REFERENCE_SAMPLE)
        tot_v += nv
        tot_t += dt
    value = tot_v / tot_t / 1e6
    sample = (f"{REFERENCE_SAMPLE}^3 corner crop of the {WORKLOAD_TEXT.split(':')[0]} field per "
              "step, standard reduction (fast mode), one thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAME,
        "data": "synthetic", "config": {"workload": WORKLOAD_TEXT, "oracle_sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample, **host_info()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


SERVE_LOADS = (0.5, 0.8, 0.95)   # Poisson arrival rates, fractions of one-at-a-time capacity


def serving_section():
    """Continuous batching vs one request at a time on the serving workload:
    fields of log-uniform shapes in [16,128]^3 (16 Gaussians + 1e-3 noise,
    float32); back to back (throughput), then Poisson arrivals at 50, 80 and
    95 % of the one-at-a-time capacity (latency, split into the wait for a
    slot and the service)."""
    from paper_2206_13932_gb300 import serve
    fields = sf.serving_fields(SERVE_REQUESTS)
    nvert = sum(f.size for f in fields)
    zeros = np.zeros(len(fields))
    serve.run_stream(fields[:8], zeros[:8], slots=4)             # warm-up
    r1, w1 = serve.run_stream(fields, zeros, slots=1)             # back to back, one at a time
    cap = len(fields) / w1
    r4, w4 = serve.run_stream(fields, zeros, slots=4)             # back to back, 4 slots
    rB, wB = serve.run_stream(fields, zeros, slots=4, max_batch=SERVE_BATCH)   # batched
    out = {
        "requests": len(fields), "mean_vertices": nvert / len(fields),
        "saturated": {"one_at_a_time_rps": cap, "one_at_a_time_Mvertices_s": nvert / w1 / 1e6,
                      "served_4_slots_rps": len(fields) / w4,
                      "served_4_slots_Mvertices_s": nvert / w4 / 1e6,
                      f"batched_4_slots_x{SERVE_BATCH}_rps": len(fields) / wB,
                      f"batched_4_slots_x{SERVE_BATCH}_Mvertices_s": nvert / wB / 1e6},
    }
    for rho in SERVE_LOADS:
        arr = sf.poisson_arrivals(len(fields), rho * cap)
        rb, _ = serve.run_stream(fields, arr, slots=4)
        rbb, _ = serve.run_stream(fields, arr, slots=4, max_batch=SERVE_BATCH)
        rs, _ = serve.run_stream(fields, arr, slots=1)
        out[f"poisson_rho_{rho}"] = {"rate_rps": rho * cap,
                                     "served_4_slots": serve.latency_stats(rb),
                                     f"batched_4_slots_x{SERVE_BATCH}": serve.latency_stats(rbb),
                                     "one_at_a_time": serve.latency_stats(rs)}
    return out


def roofline_gradient(n, s_in, stats, kavg, hbm, src):
    """The gradient stage against its algorithmic bytes: every value read once
    (N*s_in) and every critical simplex written once (8*|C|), over the device
    time of classification + compaction + ProcessLowerStars."""
    ncrit = sum(stats[f"c{d}"] for d in range(4))
    nbytes = n * s_in + 8 * ncrit
    ms = kavg["classify"] + kavg["compact"] + kavg["process_lower_stars"]
    gbs = nbytes / (ms * 1e-3) / 1e9 if ms > 0 else None
    return {"bound": "hbm", "kernel": "gradient stage (k_classify2, k_compact2, k_pls_keys, k_pls_run)",
            "achieved": gbs, "peak": hbm, "unit": "GB/s",
            "frac": gbs / hbm if gbs is not None else None, "traffic": None,
            "algorithmic_bytes_per_launch": nbytes, "ms": ms, "peak_source": src,
            "critical_simplices": ncrit,
            "note": "bound by ProcessLowerStars' integer work on the PL-critical vertices, "
                    "not by HBM"}


def roofline_classify(n, s_in, kavg, hbm, src):
    """The per-vertex stencil (k_classify2): values in, one flag byte out."""
    nbytes = n * s_in + n + 4 * (n // 2048 + 1)      # values in, flag bytes out, tile counts
    gbs = nbytes / (kavg["classify"] * 1e-3) / 1e9
    traffic = (CLASSIFY_TRAFFIC["bytes_per_launch"]
               if CLASSIFY_TRAFFIC["sources_sha256"] == _kernel_sources_sha256() else None)
    return {"bound": "hbm", "kernel": "k_classify2", "achieved": gbs, "peak": hbm,
            "unit": "GB/s", "frac": gbs / hbm, "traffic": traffic,
            "algorithmic_bytes_per_launch": nbytes, "peak_source": src}


def roofline_pls(n, stats, kavg):
    """ProcessLowerStars is bound by instruction issue (its integer work per
    star), so its roofline is the issue rate: 152 SMs x 4 schedulers x one
    warp instruction per cycle at the 2070 MHz maximum clock.  Achieved = the
    warp instructions it issues (ncu count per star x the stars of this
    launch) over its CUDA-event time; null when the kernel's code differs
    from the capture's."""
    ok = PLS_ISSUE["sources_sha256"] == _kernel_sources_sha256(_PLS_SPANS)
    crit = stats.get("critical_vertices", n)
    stars = n if (crit * 4 > n or n <= (1 << 25)) else crit     # dense or critical only
    ms = kavg["process_lower_stars"]
    peak = SMS * SMSPS * SM_MAX_MHZ * 1e6 / 1e9
    ach = PLS_ISSUE["warp_inst_per_star"] * stars / (ms * 1e-3) / 1e9 if ok and ms > 0 else None
    return {"bound": "alu", "kernel": "k_pls_keys + k_pls_run (ProcessLowerStars, stars sorted by shape)",
            "achieved": ach, "peak": peak, "unit": "G warp instructions/s",
            "frac": ach / peak if ach is not None else None, "traffic": None, "ms": ms,
            "stars": stars, "peak_source": "152 SMs x 4 schedulers x 2070 MHz",
            "note": "issue-bound: the second pass keeps its ALU pipe "
                    f"{PLS_ISSUE['alu_pipe_pct_run']} % busy (ncu); about "
                    f"{PLS_ISSUE['simt_lanes']} of the 32 lanes of an issued instruction do work "
                    "(the order of the lower links differs within a warp)"}


def roofline_trace(s_in, work, stats, kavg, hbm, src):
    """The D1 boundary trace against HBM.  Its algorithmic bytes are what the
    walks must read: per edge toggled, the gradient record (48 B), flag byte,
    value and row word (8 B) of the edge's vertex; per column, its entry
    (column map, vertex, local triangle: 9 B), the record of its vertex and
    its output slot (12 B + 1 overflow byte).  Toggles are counted on the
    device (dms_get_work)."""
    tog, cols = work["trace_toggles"], stats["d1_columns"]
    nbytes = tog * (48 + 1 + s_in + 8) + cols * (9 + 48 + 13)
    ms = kavg["d1_trace"]
    gbs = nbytes / (ms * 1e-3) / 1e9 if ms > 0 and tog > 0 else None
    return {"bound": "hbm", "kernel": "k_d1_trace (D1 boundary trace)", "achieved": gbs,
            "peak": hbm, "unit": "GB/s", "frac": gbs / hbm if gbs is not None else None,
            "traffic": None, "algorithmic_bytes_per_launch": nbytes, "ms": ms,
            "toggles": tog, "expansions": work["trace_expansions"], "columns": cols,
            "peak_source": src,
            "note": "latency-bound: each toggle's loads wait on the hash probe and heap "
                    "push of the step before it (per-thread scratch); the record gathers are "
                    "random"}


def roofline_reduce(work, stats, kavg, hbm, src):
    """The D1 reduction: the bytes its column additions read and write
    against HBM, beside the latency view -- its time over the longest chain
    of dependent additions one kernel made is the time per link of the
    critical path."""
    nbytes = stats["d1_bytes_read"] + stats["d1_bytes_written"]
    ms = kavg["d1_reduce"]
    gbs = nbytes / (ms * 1e-3) / 1e9 if ms > 0 and nbytes > 0 else None
    chain = work["d1_longest_chain"]
    return {"bound": "hbm", "kernel": "k_red_* (D1 reduction: rounds and asynchronous tail)",
            "achieved": gbs, "peak": hbm, "unit": "GB/s",
            "frac": gbs / hbm if gbs is not None else None, "traffic": None,
            "algorithmic_bytes_per_launch": nbytes, "ms": ms, "peak_source": src,
            "additions": stats["d1_additions"], "longest_chain": chain,
            "us_per_chain_addition": 1e3 * ms / chain if chain else None,
            "note": "bound by chains of dependent additions (each waits on the list its "
                    "predecessor wrote), not by bytes"}


def roofline_dominant(dom, kavg, rgrad, rcls, hbm, src, rpls=None, rtrace=None, rred=None):
    """The family with the most device time.  The stencil is measured against
    HBM, ProcessLowerStars against the issue rate; the walks, union-find
    levels and the D1 reduction have no algorithmic byte count that bounds
    them (dependent gathers, atomics and addition chains) and are reported
    with their time."""
    if dom == "classify":
        return dict(rcls)
    if dom == "process_lower_stars" and rpls is not None:
        return dict(rpls)
    if dom in ("process_lower_stars", "compact"):
        return dict(rgrad)
    if dom == "d1_trace" and rtrace is not None:
        return dict(rtrace)
    if dom == "d1_reduce" and rred is not None:
        return dict(rred)
    return {"bound": "hbm", "kernel": dom, "achieved": None, "peak": hbm, "unit": "GB/s",
            "frac": None, "traffic": None, "ms": kavg[dom], "peak_source": src,
            "note": "latency-bound (dependent loads, atomics); no algorithmic byte count"}


def run_ours(args):
    import torch
    import paper_2206_13932_gb300 as dms
    from paper_2206_13932_gb300 import replicas

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dms.build()
    shape, dtype, recipe = sf.CONFIGS[WORKLOAD]
    nx, ny, nz = shape
    n = nx * ny * nz
    field = workload_field()
    dev = torch.from_numpy(field).cuda()
    host = torch.from_numpy(field).pin_memory()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    g = dms.Grid(shape, dtype)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        g.compute(dev)
    # pinned host buffers for the pairs of the end-to-end runs (sized once)
    pcount, ecount = g.counts()
    outs = []
    for d in range(3):
        k = pcount[d] + ecount[d]
        buf = torch.empty(max(k, 1) * dms.PAIR_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
        outs.append(buf.numpy().view(dms.PAIR_DTYPE))
    # ---- device-resident timing (inputs in HBM, L2 flushed before each step)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kern = {k: 0.0 for k in g.KERNELS}
    launches = 0
    barrier()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            g.compute(dev)
            ends[k].record(stream)
            for name, ms in g.kernel_ms().items():
                kern[name] += ms
            launches += g.stats()["launches"]
        barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = replicas.max_over_ranks(sum(step_ms) / len(step_ms), device="cuda")
    value = replicas.job_throughput(n, ms) / 1e6
    stats = g.stats()
    counts = g.counts()
    stage = g.stage_ms()
    # ---- end to end through the C ABI: pinned host field in, host pairs out
    e2e_ms, comp_ms, fetch_ms, h2d_ms = [], [], [], []
    d2h = 0
    for k in range(args.warmup):             # untimed: the handle's host-input buffer
        g.compute(host)
        for d in range(3):
            g.fetch(d, out=outs[d])
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.compute(host)
        t1 = time.perf_counter()
        pairs = [g.fetch(d, out=outs[d]) for d in range(3)]
        t2 = time.perf_counter()
        e2e_ms.append(1e3 * (t2 - t0))
        comp_ms.append(1e3 * (t1 - t0))
        fetch_ms.append(1e3 * (t2 - t1))
        h2d_ms.append(g.stage_ms()["h2d"])
        d2h = sum(p.nbytes for p in pairs)
    e2e_val = replicas.job_throughput(
        n, replicas.max_over_ranks(statistics.mean(e2e_ms), device="cuda")) / 1e6
    if rank != 0:
        return
    # ---- rooflines
    kavg = {k: v / args.steps for k, v in kern.items()}
    dom = max(kavg, key=kavg.get)
    s_in = np.dtype(dtype).itemsize
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    src = "measured" if peaks else "fallback"
    rgrad = roofline_gradient(n, s_in, stats, kavg, hbm, src)
    rcls = roofline_classify(n, s_in, kavg, hbm, src)
    rpls = roofline_pls(n, stats, kavg)
    work = g.work()
    rtrace = roofline_trace(s_in, work, stats, kavg, hbm, src)
    rred = roofline_reduce(work, stats, kavg, hbm, src)
    roofline = roofline_dominant(dom, kavg, rgrad, rcls, hbm, src, rpls, rtrace, rred)
    serving = None
    if not args.no_serve:
        try:
            serving = serving_section()
        except Exception as e:   # the headline line is printed even if serving fails
            serving = {"error": f"{type(e).__name__}: {e}"}
    # oracle on a bounded crop of the same field
    nv, dt, _ = _oracle_sample(field, ORACLE_SAMPLE)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE_NAME, "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT,
                   "l2": "flushed (256 MiB write) before every timed step",
                   "parallelism": f"replicas x{ws}"},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": n * s_in,
                "d2h_bytes_per_step": d2h},
        # where an end-to-end step goes (wall clock, mean): the compute call
        # with its host-to-device copy (and that copy alone, CUDA events), then
        # the three fetches of the pairs into pinned host memory
        "e2e_split_ms": {"compute_call": statistics.mean(comp_ms),
                         "h2d_copy": statistics.mean(h2d_ms),
                         "fetch_calls": statistics.mean(fetch_ms)},
        "gpu_launches": launches,
        "roofline": roofline,
        "roofline_gradient": rgrad,
        "roofline_classify": rcls,
        "roofline_pls": rpls,
        "roofline_d1_trace": rtrace,
        "roofline_d1_reduce": rred,
        "dominant_kernel": {"name": dom, "ms": kavg[dom]},
        "kernel_ms": kavg,
        "stage_ms": stage,
        "stats": stats,
        "pairs": {"d0": counts[0][0], "d1": counts[0][1], "d2": counts[0][2],
                  "essential": list(counts[1])},
        "cpu_baseline": {"value": nv / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{ORACLE_SAMPLE}^3 corner crop of the same field, standard "
                                   "reduction (fast mode), one thread",
                         "seconds": dt, **host_info()},
        "clocks": clk.summary(),
        "serving": serving,
    }
    print(json.dumps(line))
    g.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
