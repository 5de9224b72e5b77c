"""Autotuner for the planner's knobs (hankel_set_tuning).

Times the batched forward product on the current GPU for a grid of
(pass_cost, points_per_thread) settings -- pass_cost steers the FFT lengths
and radix sequences the planner picks, points_per_thread the threads per job
-- and caches the fastest setting with the whole table in autotune.json next
to the library.  The binding applies the cached choice when it loads the
library on a device with the same name.

    python -m paper_1401_6238_gb300.autotune          # tune on the benchmark workload
"""

import json
import os
import sys
import time

from . import hankel as hk
from . import workloads as wl

GRID = [(pc, ppt) for pc in (5.0, 10.0, 20.0, 40.0) for ppt in (16, 32)]


def time_setting(batch, pass_cost, ppt, steps=20, warmup=3):
    import torch
    hk.hankel_set_tuning(pass_cost, ppt)
    plan = hk.Plan(hk.batch_descs(batch), hk.R32, hk.SAME_X)
    dev = torch.device("cuda")
    copies = 4
    Hs = [torch.tensor(batch.h, dtype=torch.float32, device=dev) for _ in range(copies)]
    Xs = [torch.tensor(batch.x, dtype=torch.float32, device=dev) for _ in range(copies)]
    Y = torch.zeros(batch.y_len, dtype=torch.float32, device=dev)
    for i in range(warmup):
        plan.txv(Hs[i % copies], Xs[i % copies], Y)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for i in range(steps):
        plan.txv(Hs[i % copies], Xs[i % copies], Y)
    b.record()
    torch.cuda.synchronize()
    info = plan.info
    plan.close()
    return a.elapsed_time(b) / steps, info


def tune(batch=None, grid=GRID, path=hk.TUNING_PATH):
    import torch
    hk.load()
    batch = batch if batch is not None else wl.batched_square(count=8192, seed=1)
    old = hk.hankel_get_tuning()
    rows = []
    for pc, ppt in grid:
        ms, info = time_setting(batch, pc, ppt)
        rows.append({"pass_cost": pc, "points_per_thread": ppt, "ms_per_step": ms,
                     "distinct_lengths": info["distinct_lengths"], "sum_length": info["sum_length"]})
    best = min(rows, key=lambda r: r["ms_per_step"])
    hk.hankel_set_tuning(*old)
    rec = {"device": torch.cuda.get_device_name(), "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()),
           "workload": "8192 square real tensors, m in {3,4,5}, n in [16,1024], FP32 forward",
           "best": {"pass_cost": best["pass_cost"], "points_per_thread": best["points_per_thread"]},
           "results": rows}
    if path:
        with open(path, "w") as f:
            json.dump(rec, f, indent=1)
    return rec


if __name__ == "__main__":
    out = tune(path=sys.argv[1] if len(sys.argv) > 1 else hk.TUNING_PATH)
    print(json.dumps(out["best"]), file=sys.stderr)
    for r in out["results"]:
        print(r, file=sys.stderr)
