"""Autotuner for the planner's choices.

Two tables, cached in autotune.json next to the library and applied by the
binding when it loads the library on a device with the same name:

* the per-length launches' knobs (hankel_set_tuning): the batched forward
  product timed for a grid of (pass_cost, points_per_thread) settings --
  pass_cost steers the FFT lengths and radix sequences the planner picks,
  points_per_thread the threads per job;
* the per-bin policy (hankel_set_bin_policy), for each FFT-length bin of
  the persistent kernel: which path is faster for the bin's tensors (the
  persistent launch or the per-length launches, both timed on a batch of
  the bin), and from which order m FP64 spectrum powers pay: the FP32
  error with and without them, for m = 2 .. 8, measured against the
  library's FP64 path (which the tests hold to the FP64 oracle at 1e-12)
  on unscaled Gaussian inputs.  FP64 powers are chosen for m >= m0 only
  when they cut the largest FP32 error by a quarter or more for every
  order from m0 up and the FP32 error is above half the 1e-5 bound.

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


BINS = [32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048, 3072, 4096, 5120]
TOL32 = 1e-5


def bin_batch(L, orders, count, seed, scaled=True):
    """``count`` square real tensors whose generating length d falls in the
    bin of L (above the previous bin), orders drawn from ``orders`` (those
    that reach the bin)."""
    import numpy as np
    lo = BINS[BINS.index(L) - 1] if L != BINS[0] else 0
    rng = np.random.default_rng(seed)
    cand = [(m, n) for m in orders for n in range(2, L + 1) if lo < m * (n - 1) + 1 <= L]
    if not cand:
        return None
    pick = [cand[i] for i in rng.integers(0, len(cand), size=count)]
    hs, xs = [], []
    for m, n in pick:
        d = m * (n - 1) + 1
        h, x = rng.standard_normal(d), rng.standard_normal(n)
        if scaled:
            h, x = h / np.sqrt(d), x / np.linalg.norm(x)
        hs.append(h)
        xs.append(x)
    return wl.pack_square([m for m, _ in pick], [n for _, n in pick], hs, xs)


def _forward(batch, dtype, flags=hk.SAME_X):
    import torch
    tdt = torch.float32 if dtype == hk.R32 else torch.float64
    plan = hk.Plan(hk.batch_descs(batch), dtype, flags)
    dev = torch.device("cuda")
    H, X = torch.tensor(batch.h, dtype=tdt, device=dev), torch.tensor(batch.x, dtype=tdt, device=dev)
    Y = torch.zeros(batch.y_len, dtype=tdt, device=dev)
    plan.txv(H, X, Y)
    torch.cuda.synchronize()
    info = plan.info
    plan.close()
    return Y.double().cpu().numpy(), info


def _max_rel_err(batch, y, ref):
    import numpy as np
    return max(float(np.max(np.abs(y[o:o + n] - ref[o:o + n])) / np.max(np.abs(ref[o:o + n])))
               for o, n in zip(batch.y_off, batch.dims))


def fp64_threshold(err32, err64, tol=TOL32):
    """The smallest order m0 such that FP64 powers pay for every measured
    order m >= m0 (cut the largest FP32 error by a quarter or more, where
    that error is above half the bound); 99 (never) when the largest
    measured order already does not."""
    m0 = 99
    for m in sorted(err32, reverse=True):
        if not (err64[m] <= 0.75 * err32[m] and err32[m] > 0.5 * tol):
            break
        m0 = m
    return m0


def tuning_record():
    """The planner choices in force (knobs and per-bin policy) and the cache
    file they came from, for the benchmark line."""
    import torch
    rec = {"knobs": dict(zip(("pass_cost", "points_per_thread"), hk.hankel_get_tuning())),
           "bins": {str(L): dict(zip(("path", "fp64_from_m"), hk.hankel_get_bin_policy(L))) for L in BINS}}
    try:
        cache = json.load(open(hk.TUNING_PATH))
        if cache.get("device") == torch.cuda.get_device_name():
            rec["file"] = os.path.relpath(hk.TUNING_PATH, os.path.dirname(os.path.dirname(hk.TUNING_PATH)))
            rec["when"] = cache.get("when")
            rec["bins_when"] = cache.get("bins_when")
    except Exception:
        rec["file"] = None
    return rec


def tune_bins(batch=None, points=1 << 22, path=hk.TUNING_PATH):
    """Per-bin path and FP64-power choices; merged into the cache file.

    A bin moves to the per-length launches only when that makes the whole
    workload (``batch``, default the benchmark's) more than 2% faster: a
    bin's own batch may favour them while in the workload the bin's few
    tensors would add a launch.  Each bin is also timed alone on both paths
    (recorded, not used)."""
    import numpy as np
    import torch
    hk.load()
    batch = batch if batch is not None else wl.batched_square(count=8192, seed=1)
    dw = batch.orders * (batch.dims - 1) + 1
    old = {L: hk.hankel_get_bin_policy(L) for L in BINS}
    knobs = hk.hankel_get_tuning()
    rows = []
    try:
        hk.hankel_set_bin_policy({})
        base = time_setting(batch, *knobs)[0]
        for L in BINS:
            lo = BINS[BINS.index(L) - 1] if L != BINS[0] else 0
            in_work = int(np.count_nonzero((dw > lo) & (dw <= L)))
            hk.hankel_set_bin_policy({})
            b = bin_batch(L, (3, 4, 5), max(64, min(4096, points // L)), seed=L)
            if b is None:
                b = bin_batch(L, (2,), max(64, min(4096, points // L)), seed=L)
            ms = {}
            for p in (0, 1):
                hk.hankel_set_bin_policy({L: (p, 99)})
                ms[p] = time_setting(b, *knobs)[0]
            mixed = None
            if in_work:
                hk.hankel_set_bin_policy({L: (1, 99)})
                mixed = time_setting(batch, *knobs)[0]
            # FP32 error with and without FP64 powers, against the FP64 path
            err32, err64 = {}, {}
            for m in range(2, 9):
                e = bin_batch(L, (m,), 8, seed=100 * L + m, scaled=False)
                if e is None:
                    continue
                ref, _ = _forward(e, hk.R64)
                hk.hankel_set_bin_policy({L: (0, 99)})
                err32[m] = _max_rel_err(e, _forward(e, hk.R32)[0], ref)
                hk.hankel_set_bin_policy({L: (0, 2)})
                err64[m] = _max_rel_err(e, _forward(e, hk.R32)[0], ref)
            m0 = fp64_threshold(err32, err64)
            rows.append({"L": L, "path": 1 if mixed is not None and mixed < 0.98 * base else 0, "fp64_from_m": m0,
                         "workload_tensors": in_work, "workload_ms": base, "workload_ms_per_length": mixed,
                         "alone_tensors": len(b), "alone_persistent_ms": ms[0], "alone_per_length_ms": ms[1],
                         "err_fp32": {str(k): v for k, v in err32.items()},
                         "err_fp64_power": {str(k): v for k, v in err64.items()}})
    finally:
        hk.hankel_set_bin_policy({})
        hk.hankel_set_bin_policy({L: old[L] for L in BINS})
    if path:
        rec = json.load(open(path)) if os.path.exists(path) else {}
        if rec.get("device") != torch.cuda.get_device_name():
            rec = {"device": torch.cuda.get_device_name()}
        rec["bins_when"] = time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())
        rec["bins_workload"] = ("path: the 8192-tensor benchmark batch with the bin on each path; alone: up to 4096 "
                                "square real tensors with d in the bin, m in {3,4,5}; error: 8 unscaled Gaussian "
                                "tensors per order m = 2..8 against the FP64 path")
        rec["bins"] = rows
        with open(path, "w") as f:
            json.dump(rec, f, indent=1)
    return rows


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
        if os.path.exists(path):
            prev = json.load(open(path))
            if prev.get("device") == rec["device"]:
                for k in ("bins", "bins_when", "bins_workload"):
                    if k in prev:
                        rec[k] = prev[k]
        with open(path, "w") as f:
            json.dump(rec, f, indent=1)
    return rec


if __name__ == "__main__":
    path = sys.argv[1] if len(sys.argv) > 1 else hk.TUNING_PATH
    out = tune(path=path)
    print(json.dumps(out["best"]), file=sys.stderr)
    for r in out["results"]:
        print(r, file=sys.stderr)
    for r in tune_bins(path=path):
        print({k: r[k] for k in ("L", "path", "fp64_from_m", "workload_tensors", "workload_ms", "workload_ms_per_length",
                                 "alone_persistent_ms", "alone_per_length_ms")}, file=sys.stderr)
