"""Runs the pipeline on one synthetic field (for profiling and timing): the
driver of the ncu captures summarised under profiles/.

    python -m tests.run_case --workload noise --edge 128 [--repeat 1]

Workloads: noise (iid U[0,1) float32, seed 2), mixture_u16 (the 512^3 uint16 recipe at
the given edge), mixture32 (16 Gaussians + 1e-3 noise float32, seed 1).
"""
from __future__ import annotations

import argparse
import json
import os
import sys


def main():
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch

    import paper_2206_13932_gb300 as dms
    import synthfields as sf

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="noise", choices=["noise", "mixture_u16", "mixture32"])
    ap.add_argument("--edge", type=int, default=128)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--d1-mode", type=int, default=0)
    ap.add_argument("--op", default="diagram", choices=["diagram", "classify"],
                    help="classify: only dms_classify_static (allocates nothing but the outputs)")
    a = ap.parse_args()
    e = a.edge
    if a.workload == "noise":
        v = sf.white_noise((e, e, e), 2)
    elif a.workload == "mixture_u16":
        v = sf.config_field("mixture512_u16", shape_xyz=(e, e, e), device="cuda")
    else:
        v = sf.config_field("mixture32_f32", shape_xyz=(e, e, e))
    t = torch.from_numpy(v).cuda()
    if a.op == "classify":
        flags = torch.empty(t.numel(), dtype=torch.uint8, device="cuda")
        crit = torch.empty(t.numel(), dtype=torch.int32, device="cuda")
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = []
        for _ in range(a.repeat):
            start.record()
            n = dms.classify_static(t, flags, crit)
            end.record()
            torch.cuda.synchronize()
            ms.append(start.elapsed_time(end))
        print(json.dumps({"critical_vertices": n, "classify_call_ms": ms}))
        return
    with dms.Grid((e, e, e), v.dtype, d1_mode=a.d1_mode) as g:
        for _ in range(a.repeat):
            g.compute(t)
        print(json.dumps({"kernel_ms": g.kernel_ms(), "stage_ms": g.stage_ms(),
                          "stats": g.stats(), "counts": g.counts()}))


if __name__ == "__main__":
    main()
