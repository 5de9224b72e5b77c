"""Benchmark: batched fast Hankel tensor-vector products on GB300.

Workload (one step): 8192 independent square real Hankel tensors, order m
uniform in {3,4,5}, dimension n uniform in [16,1024], h ~ N(0,1/d),
x unit-norm Gaussian, FP32 (twiddles generated in FP64), y = H x^{m-1} for
every tensor in one hankel_txv() call.  Inputs are resident in HBM; each
timed step uses the next of several input copies (together > 4x L2) so the
step reads HBM, not L2.

Reported (one JSON line on rank 0):
  value        products/s over all ranks (device-timed, CUDA events)
  e2e          the same through hankel_txv_host() with pinned host buffers
               (H2D of h, x and D2H of y inside the timed region)
  roofline     algorithmic bytes 4*(d + 2n) per tensor / step time vs the
               measured HBM copy bandwidth
  fp64_plain   the plain FP64 path, one tensor per kernel launch, and the
               FP32/FP64 output agreement
  cpu_baseline the FP64 oracle on the host cores over a bounded sample
  accuracy     per-tensor relative infinity-norm error of the timed FP32
               output against the FP64 oracle, over every tensor of the batch
               (max and median)
--impl reference times the FP64 oracle alone (the CPU arm).
"""

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H·x^{m-1} products/s and % HBM roofline, batched FP32 vs plain FP64, same error"
WORKLOAD = {"workload": "batched square real Hankel tensors",
            "tensors": 8192, "orders": [3, 4, 5], "n_range": [16, 1024],
            "h": "N(0,1/d)", "x": "unit-norm Gaussian", "product": "y = H x^{m-1}"}


def bench_config(batch, copies):
    """The workload's description, printed by both arms."""
    return dict(WORKLOAD, l2="each step reads one of %d input copies (%.0f MB together, > 4x L2)"
                % (copies, copies * (batch.h.nbytes + batch.x.nbytes) / 2e6),
                parallelism="replicas: each rank its own 8192-tensor batch")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


_BATCH = {}


def oracle_sample_worker(args):
    lo, hi, seed = args
    import oracle
    from paper_1401_6238_gb300 import workloads as wl
    if seed not in _BATCH:
        _BATCH[seed] = wl.batched_square(count=8192, seed=seed)
    b = _BATCH[seed]
    for i in range(lo, hi):
        m, n, h, x = b.tensor(i)
        oracle.fast_y(h, [x] * (m - 1), [n] * m)
    return hi - lo


def oracle_refs_worker(args):
    """Oracle outputs y (FP64) of tensors lo .. hi-1 of the seeded batch."""
    lo, hi, seed = args
    import oracle
    from paper_1401_6238_gb300 import workloads as wl
    if seed not in _BATCH:
        _BATCH[seed] = wl.batched_square(count=8192, seed=seed)
    b = _BATCH[seed]
    out = []
    for i in range(lo, hi):
        m, n, h, x = b.tensor(i)
        out.append(oracle.fast_y(h, [x] * (m - 1), [n] * m).real)
    return out


def oracle_errors(batch, y, seed, pool):
    """Per-tensor ||y_i - y_i^oracle||_inf / ||y_i^oracle||_inf over the batch."""
    chunk = 64
    tasks = [(lo, min(len(batch), lo + chunk), seed) for lo in range(0, len(batch), chunk)]
    refs = [r for part in pool.map(oracle_refs_worker, tasks) for r in part]
    err = np.empty(len(batch))
    for i, ref in enumerate(refs):
        o, n = batch.y_off[i], batch.dims[i]
        err[i] = np.max(np.abs(y[o:o + n] - ref)) / np.max(np.abs(ref))
    return err


def cpu_oracle(seconds=12.0, seed=1, pool=None, cores=1):
    """Time the FP64 oracle (own radix-2 FFT embedding) on the host cores over
    a bounded sample of the workload; returns products/s."""
    chunk = 16
    done = 0
    t0 = time.perf_counter()
    nxt = 0
    while time.perf_counter() - t0 < seconds and nxt < 8192:
        tasks = []
        for _ in range(cores):
            if nxt >= 8192:
                break
            tasks.append((nxt, min(8192, nxt + chunk), seed))
            nxt += chunk
        if pool is not None:
            done += sum(pool.map(oracle_sample_worker, tasks))
        else:
            done += sum(oracle_sample_worker(t) for t in tasks)
    dt = time.perf_counter() - t0
    return done / dt, done, dt


def start_clock_sampler(path):
    try:
        return subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
             "--format=csv,noheader,nounits", "-lms", "200"],
            stdout=open(path, "w"), stderr=subprocess.DEVNULL)
    except Exception:
        return None


def read_clocks(path, proc, gpu_index):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except Exception:
        proc.kill()
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9 or f[0] != str(gpu_index):
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
    except OSError:
        return None
    if not sm:
        return None
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
            "samples": len(sm), "window": "%.1f s soak of the same step just before the timed region, and the "
                                          "timed region" % SOAK_SECONDS}


def rank_seed(rank):
    """Each rank benchmarks its own batch (weak scaling): seed 1 + rank."""
    return 1 + int(rank)


def max_over_ranks(value, dist, device):
    """Largest value over all ranks (a step time): the job's wall time."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world, per_rank_units, seconds):
    """Whole-job throughput: units processed by all ranks / slowest rank's time."""
    return world * per_rank_units / seconds


def profiled_traffic():
    """DRAM bytes per step of the forward kernel from the committed ncu
    capture, or None when the kernel sources changed since it was taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "fast_fwd_traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
        h = hashlib.sha256()
        for f in rec["sources"]:
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(fh.read())
        return rec["bytes_per_step"] if h.hexdigest() == rec["sources_sha256"] else None
    except Exception:
        return None


FP32_LANES_PER_SM = 128
# untimed run of the step under the clock sampler before the timed region
SOAK_SECONDS = 0.8


def alu_roofline(flops, kernel_ms, clocks, sms):
    """FP32 CUDA-core roofline of the forward step (flops per step / kernel
    time against 2 x lanes x SMs x the median sampled SM clock); ``sms`` is
    the device's multiprocessor count."""
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    peak = 2.0 * FP32_LANES_PER_SM * sms * mhz * 1e6 / 1e12
    achieved = flops / (kernel_ms / 1000.0) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "flops_per_step": flops,
            "peak_source": "derived: %d SMs (device multiprocessor count) x 128 FP32 lanes x 2 x %.0f MHz "
                           "(median sampled SM clock)" % (sms, mhz)}


def timed(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def sec_grad(dev, stream, steps, warmup):
    import torch
    from paper_1401_6238_gb300 import hankel as hk
    from paper_1401_6238_gb300 import workloads as wl
    f32 = lambda a: torch.tensor(a, dtype=torch.float32, device=dev)
    c64 = lambda a: torch.tensor(a, dtype=torch.complex64, device=dev)
    out = {}
    # gradient workload: loss through y = H x^{m-1}, m = 4, n = 4096, batch 64
    b = wl.grad_case(batch=64, m=4, n=4096, seed=3)
    plan = hk.Plan(hk.batch_descs(b), hk.R32, hk.SAME_X | hk.STORE_SPECTRA)
    H, X = f32(b.h), f32(b.x)
    Y = torch.zeros(plan.info["y_elems"], dtype=torch.float32, device=dev)
    G = f32(np.random.default_rng(0).standard_normal(plan.info["y_elems"]))
    gh, gx = torch.zeros_like(H), torch.zeros_like(X)

    def grad_step():
        plan.txv(H, X, Y, None, stream)
        plan.backward(G, H, X, gh, gx, stream)

    ms = timed(grad_step, steps, warmup, stream)
    out["grad"] = {"workload": "m=4, n=4096 (d=16381, L=16384), batch 64, FP32 forward + backward (spectra kept)",
                   "value": 64 / (ms / 1e3), "unit": "forward+backward products/s", "ms_per_step": ms}
    plan.close()
    return out


def sec_batch_adjoint(dev, stream, steps, warmup):
    import torch
    from paper_1401_6238_gb300 import hankel as hk
    from paper_1401_6238_gb300 import workloads as wl
    out = {}
    # adjoint of the benchmark batch: grad_h and grad_x of <g, y> for the
    # 8192 tensors (spectra recomputed, not kept from a forward call)
    b = wl.batched_square(count=8192, seed=1)
    plan = hk.Plan(hk.batch_descs(b), hk.R32, hk.SAME_X)
    H = torch.tensor(b.h, dtype=torch.float32, device=dev)
    X = torch.tensor(b.x, dtype=torch.float32, device=dev)
    G = torch.tensor(np.random.default_rng(0).standard_normal(b.y_len), dtype=torch.float32, device=dev)
    gh, gx = torch.zeros_like(H), torch.zeros_like(X)
    ms = timed(lambda: plan.backward(G, H, X, gh, gx, stream), steps, warmup, stream)
    # read g, h, x and write grad_h, grad_x: 4 (2 d + 3 n) bytes per tensor
    alg = float(sum(4 * (2 * (m * (n - 1) + 1) + 3 * n) for m, n in zip(b.orders, b.dims)))
    out["batch_adjoint"] = {"workload": "adjoint of the 8192-tensor batch (grad_h, grad_x of <g, y>), FP32, spectra "
                                        "recomputed", "value": len(b) / (ms / 1e3), "unit": "adjoint products/s",
                            "ms_per_step": ms, "algorithmic_bytes": alg,
                            "achieved_gbs": alg / (ms / 1e3) / 1e9, "launches": plan.info["backward_launches"]}
    plan.close()
    return out


def sec_hooi_products(dev, stream, steps, warmup):
    import torch
    from paper_1401_6238_gb300 import hankel as hk
    from paper_1401_6238_gb300 import workloads as wl
    f32 = lambda a: torch.tensor(a, dtype=torch.float32, device=dev)
    c64 = lambda a: torch.tensor(a, dtype=torch.complex64, device=dev)
    out = {}
    # HOOI tensor-matrix products: 16 x 16 column pairs, shared h, complex64
    R, N = 16, 4094
    s = wl.edf_1d_signal(N=N, seed=4)
    dims = [N + 2 - 2 * ((N + 2) // 3), (N + 2) // 3, (N + 2) // 3]
    U = wl.unit_columns(dims[1], R, seed=5)
    V = wl.unit_columns(dims[2], R, seed=6)
    descs = hk.make_descs(R * R)
    for k in range(R * R):
        i, j = divmod(k, R)
        descs[k]["m"] = 3
        descs[k]["n"][:3] = dims
        descs[k]["x_off"][1] = i * dims[1]
        descs[k]["x_off"][2] = R * dims[1] + j * dims[2]
        descs[k]["y_off"] = k * dims[0]
    plan = hk.Plan(descs, hk.C64, 0)
    Hs, Xs = c64(s), c64(np.concatenate([U.T.reshape(-1), V.T.reshape(-1)]))
    Ys = torch.zeros(R * R * dims[0], dtype=torch.complex64, device=dev)
    ms = timed(lambda: plan.txv(Hs, Xs, Ys, None, stream), steps, warmup, stream)
    out["hooi_products"] = {"workload": "complex64 order-3 Hankel of a length-4094 exponential signal "
                                        "(1366 x 1365 x 1365), 16 x 16 column pairs H x2 u_i x3 v_j",
                            "value": R * R / (ms / 1e3), "unit": "products/s", "ms_per_step": ms}
    plan.close()
    return out


def sec_bhhb(dev, stream, steps, warmup):
    import torch
    from paper_1401_6238_gb300 import hankel as hk
    from paper_1401_6238_gb300 import workloads as wl
    f32 = lambda a: torch.tensor(a, dtype=torch.float32, device=dev)
    c64 = lambda a: torch.tensor(a, dtype=torch.complex64, device=dev)
    out = {}
    # 2D block (BHHB) products: 256 x 256 signal, blocks 86^3 x 86^3, 32 triples
    count = 32
    S = wl.edf_2d_signal(seed=5)
    Xb = wl.unit_matrices(2 * count, 86, 86, seed=6)
    descs = hk.make_descs(count)
    for t in range(count):
        descs[t]["m"] = 3
        descs[t]["n"][:3] = 86
        descs[t]["N"][:3] = 86
        descs[t]["x_off"][1] = (2 * t) * 86 * 86
        descs[t]["x_off"][2] = (2 * t + 1) * 86 * 86
        descs[t]["y_off"] = t * 86 * 86
    plan = hk.Plan(descs, hk.C64, hk.BLOCK)
    Hb = c64(S.reshape(-1, order="F"))
    Xv = c64(np.concatenate([X.reshape(-1, order="F") for X in Xb]))
    Yb = torch.zeros(count * 86 * 86, dtype=torch.complex64, device=dev)
    Gb = c64(np.random.default_rng(1).standard_normal(count * 86 * 86))
    ghb, gxb = torch.zeros_like(Hb), torch.zeros_like(Xv)
    ms_f = timed(lambda: plan.txv_block(Hb, Xv, Yb, None, stream), steps, warmup, stream)
    ms_b = timed(lambda: plan.backward(Gb, Hb, Xv, ghb, gxb, stream), steps, warmup, stream)
    out["bhhb"] = {"workload": "complex64 256 x 256 2D exponential signal, BHHB blocks (86,86,86) x (86,86,86), "
                               "32 vector triples, forward and adjoint",
                   "value": count / ((ms_f + ms_b) / 1e3), "unit": "forward+adjoint products/s",
                   "forward_ms": ms_f, "adjoint_ms": ms_b}
    plan.close()
    return out


def sec_distinct(dev, stream, steps, warmup):
    import torch
    from paper_1401_6238_gb300 import hankel as hk
    from paper_1401_6238_gb300 import workloads as wl
    f32 = lambda a: torch.tensor(a, dtype=torch.float32, device=dev)
    c64 = lambda a: torch.tensor(a, dtype=torch.complex64, device=dev)
    out = {}
    # distinct vectors per mode (Section 3's m + 1 transform form): the
    # 8192-tensor batch shape with x_1 .. x_m per tensor, FP32
    bd, xoffs = wl.batched_distinct(8192, seed=12)
    dd = hk.make_descs(len(bd))
    dd["m"] = bd.orders
    for p in range(hk.MAX_ORDER):
        dd["n"][:, p] = np.where(p < bd.orders, bd.dims, 0)
    dd["h_off"] = bd.h_off
    for i, offs in enumerate(xoffs):
        dd["x_off"][i, :len(offs)] = offs
    dd["y_off"] = bd.y_off
    plan = hk.Plan(dd, hk.R32, 0)
    Hd, Xd = f32(bd.h), f32(bd.x)
    Yd = torch.zeros(bd.y_len, dtype=torch.float32, device=dev)
    Ad = torch.zeros(len(bd), dtype=torch.float32, device=dev)
    ms_y = timed(lambda: plan.txv(Hd, Xd, Yd, None, stream), steps, warmup, stream)
    ms_ya = timed(lambda: plan.txv(Hd, Xd, Yd, Ad, stream), steps, warmup, stream)
    out["distinct"] = {"workload": "8192 real tensors, m in {3,4,5}, n in [16,1024], a different unit-norm vector "
                                   "in every mode, FP32; y = H x_2 ... x_m, and with alpha = H x_1 ... x_m",
                       "value": len(bd) / (ms_y / 1e3), "unit": "products/s", "y_ms": ms_y, "y_and_alpha_ms": ms_ya,
                       "jobs": plan.info["jobs"], "launches": plan.info["launches"]}
    plan.close()
    return out


def sec_level3(dev, stream, steps, warmup):
    import torch
    from paper_1401_6238_gb300 import hankel as hk
    from paper_1401_6238_gb300 import workloads as wl
    f32 = lambda a: torch.tensor(a, dtype=torch.float32, device=dev)
    c64 = lambda a: torch.tensor(a, dtype=torch.complex64, device=dev)
    out = {}
    # level-3 block Hankel products (Section 2.2): a 64^3 3D signal as
    # generating tensor, sizes (22,22,22) at every level, 32 vector triples
    count, n3 = 32, 22 ** 3
    S3 = wl.edf_3d_signal(seed=10)
    X3 = wl.random_arrays(2 * count, (22, 22, 22), seed=11)
    d3 = hk.level_descs([[22, 22, 22]] * 3, [0] * count, [[0, 2 * t * n3, (2 * t + 1) * n3] for t in range(count)],
                        [t * n3 for t in range(count)])
    plan = hk.Plan(d3, hk.C64, 0)
    H3 = c64(S3.reshape(-1, order="F"))
    Xv3 = c64(np.concatenate([X.reshape(-1, order="F") for X in X3]))
    Y3 = torch.zeros(count * n3, dtype=torch.complex64, device=dev)
    G3 = c64(np.random.default_rng(2).standard_normal(count * n3))
    gh3, gx3 = torch.zeros_like(H3), torch.zeros_like(Xv3)
    ms_f = timed(lambda: plan.txv_block(H3, Xv3, Y3, None, stream), steps, warmup, stream)
    ms_b = timed(lambda: plan.backward(G3, H3, Xv3, gh3, gx3, stream), steps, warmup, stream)
    out["level3"] = {"workload": "complex64 level-3 block Hankel, generating tensor a 64^3 3D exponential signal, "
                                 "sizes (22,22,22) at each level (modes of 10648), 32 vector triples, forward and adjoint",
                     "value": count / ((ms_f + ms_b) / 1e3), "unit": "forward+adjoint products/s",
                     "forward_ms": ms_f, "adjoint_ms": ms_b, "launches": plan.info["launches"],
                     "workspace_bytes": plan.info["workspace_bytes"]}
    plan.close()
    return out


SECONDARY = {"grad": sec_grad, "batch_adjoint": sec_batch_adjoint, "hooi_products": sec_hooi_products,
             "bhhb": sec_bhhb, "distinct": sec_distinct,
             "level3": sec_level3}


def secondary_workloads(dev, stream, steps=10, warmup=3, only=None):
    """The other workloads of the path, timed on the device (inputs resident;
    these batches are L2-sized, so they measure the kernels, not HBM);
    ``only`` names a subset (SECONDARY keys and "edf")."""
    out = {}
    for name, fn in SECONDARY.items():
        if only is None or name in only:
            out.update(fn(dev, stream, steps, warmup))
    if only is None or "edf" in only:
        out.update(edf_workloads(dev, stream))
    return out


def edf_workloads(dev, stream):
    """Exponential data fitting (Section 4): HOOI sweeps (Algorithm 4.1) on the
    length-4094 1D signal and HOTF sweeps (Algorithm 4.2) on the 256 x 256 2D
    signal.  A sweep is the batched products of every mode update plus the
    QR/SVD of each unfolding (torch.linalg) on the same stream."""
    import time
    import torch
    from paper_1401_6238_gb300 import edf
    from paper_1401_6238_gb300 import hankel as hk
    from paper_1401_6238_gb300 import workloads as wl
    out = {}
    s1 = wl.edf_1d_signal(N=4094, K=8, seed=4)
    S2 = wl.edf_2d_signal(seed=5)
    cases = [("edf_1d_R8", s1, 8, None), ("edf_1d_R16", s1, 16, None), ("edf_2d_R12", S2, 12, 86)]
    for name, sig, R, blk in cases:
        if blk is None:
            T = edf.HankelTensor(sig, edf.hankel_dims(sig.size), dtype=hk.C64, device=dev)
            h = edf.HOOI(T, R)
            work = "complex64 order-3 Hankel 1366 x 1365 x 1365 (N = 4094, K = 8, 20 dB), Algorithm 4.1, R = %d" % R
        else:
            T = edf.HankelTensor(sig, [blk] * 3, [blk] * 3, dtype=hk.C64, device=dev)
            h = edf.HOOI(T, R, symmetric=True)
            work = ("complex64 order-3 BHHB, blocks (86,86,86) x (86,86,86) of a 256 x 256 signal (K = 12, 20 dB), "
                    "Algorithm 4.2, R = %d" % R)
        h.init()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.init()
        torch.cuda.synchronize()
        init_ms = (time.perf_counter() - t0) * 1e3
        modes = list(h.plans)
        products = sum(h.Y[p].numel() // T.sizes[p] for p in modes)
        ms_prod = timed(lambda: [T.run(h.plans[p], h.X, h.Y[p]) for p in modes], 10, 3, stream)
        ms_sweep = timed(h.sweep, 5, 2, stream)
        out[name] = {"workload": work, "value": 1e3 / ms_sweep, "unit": "sweeps/s", "ms_per_sweep": ms_sweep,
                     "products_per_sweep": products, "products_ms_per_sweep": ms_prod, "init_ms": init_ms,
                     "fit_50_sweeps_ms": init_ms + 50 * ms_sweep}
        h.close()
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import multiprocessing as mp
    from paper_1401_6238_gb300 import workloads as wl
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        per_step = max(5.0, 60.0 / max(1, args.steps + args.warmup))
        for _ in range(args.warmup):
            cpu_oracle(seconds=min(per_step, 5.0), pool=pool, cores=cores)
        vals = []
        for _ in range(args.steps):
            v, n, dt = cpu_oracle(seconds=per_step, pool=pool, cores=cores)
            vals.append((v, n, dt))
    value = float(np.mean([v[0] for v in vals]))
    total_n = sum(v[1] for v in vals)
    ms = 1000.0 * 8192 / value
    line = {"metric": METRIC, "value": value, "unit": "products/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": bench_config(wl.batched_square(count=8192, seed=rank_seed(0)), max(2, args.copies)),
            "cpu_baseline": {"value": value, "unit": "products/s", "cores": cores, "kind": "oracle",
                             "sample": "%d tensors of the 8192-tensor workload (FP64 radix-2 embedding FFT, "
                                       "spawn pool of %d processes), %d steps" % (total_n, cores, args.steps)},
            "e2e": {"value": value, "unit": "products/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--copies", type=int, default=6)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-secondary", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--secondary", default=None,
                    help="comma-separated secondary workloads to run alone (grad, batch_adjoint, hooi_products, bhhb, "
                         "distinct, level3, edf); prints their JSON and exits")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.secondary:
        import torch
        torch.cuda.set_device(0)
        only = [w.strip() for w in args.secondary.split(",") if w.strip()]
        res = secondary_workloads(torch.device("cuda", 0), torch.cuda.current_stream(), args.steps, args.warmup, only)
        print(json.dumps({"secondary": res}))
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    # the CPU baseline's process pool starts before the first GPU call
    pool = None
    cores = os.cpu_count() or 1
    if rank == 0 and world == 1 and not args.no_cpu:
        import multiprocessing as mp
        pool = mp.get_context("spawn").Pool(cores)

    import torch
    from paper_1401_6238_gb300 import hankel as hk
    from paper_1401_6238_gb300 import workloads as wl

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    # each rank processes its own full batch (weak scaling: fixed work per GPU)
    batch = wl.batched_square(count=8192, seed=rank_seed(rank))
    descs = hk.batch_descs(batch)
    plan = hk.Plan(descs, hk.R32, hk.SAME_X)
    info = plan.info
    from paper_1401_6238_gb300 import autotune
    tuning = autotune.tuning_record()
    copies = max(2, args.copies)
    Hs = [torch.tensor(batch.h, dtype=torch.float32, device=dev) for _ in range(copies)]
    Xs = [torch.tensor(batch.x, dtype=torch.float32, device=dev) for _ in range(copies)]
    Ys = [torch.zeros(batch.y_len, dtype=torch.float32, device=dev) for _ in range(copies)]
    stream = torch.cuda.current_stream()

    def step(i):
        c = i % copies
        plan.txv(Hs[c], Xs[c], Ys[c], None, stream)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    # per-run clock samples; BENCH_CLOCKS_CSV keeps them at a chosen path.
    # nvidia-smi samples every 200 ms and the timed steps last milliseconds,
    # so the samples cover a soak of the same step run on every rank right
    # before the timed region, and the timed region itself
    clk_path = os.environ.get("BENCH_CLOCKS_CSV") or os.path.join(
        tempfile.gettempdir(), "bench_clocks_%d.csv" % os.getpid())
    sampler = start_clock_sampler(clk_path) if rank == 0 else None
    soak_end = time.perf_counter() + SOAK_SECONDS
    i = args.warmup
    while time.perf_counter() < soak_end:
        for _ in range(25):
            step(i)
            i += 1
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(args.steps):
        ev[i][0].record(stream)
        step(args.warmup + i)
        ev[i][1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    clocks = read_clocks(clk_path, sampler, local) if rank == 0 else None
    total_ms = t_start.elapsed_time(t_end)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = max_over_ranks(total_ms / args.steps, dist, dev)
    value = aggregate_rate(world, len(batch), ms / 1000.0)

    # roofline of the forward kernel: algorithmic bytes per step / kernel time
    alg_bytes = float(sum(4 * (m * (n - 1) + 1 + 2 * n) for m, n in zip(batch.orders, batch.dims)))
    peak, peak_src = peaks()
    kernel_ms = float(np.mean(step_ms))
    achieved = alg_bytes / (kernel_ms / 1000.0) / 1e9
    traffic = profiled_traffic()
    # the same step against the FP32 CUDA-core roofline: 5 L log2 L flops per
    # complex length-L transform, three transforms per pair of tensors (1.5
    # per tensor); the spectrum products are not counted.  Peak: 152 SMs x
    # 128 FP32 lanes x 2 flops (FMA) x the SM clock sampled during the run.
    lens = [hk.hankel_fft_length(int(m * (n - 1) + 1)) for m, n in zip(batch.orders, batch.dims)]
    alg_flops = float(sum(1.5 * 5.0 * L * np.log2(L) for L in lens))

    # the same step replayed from a CUDA graph (the launches and the plan's
    # stream fork/join captured once)
    graph, local_gms = None, float("inf")  # inf: this rank has no replay time
    try:
        gs = torch.cuda.Stream()
        gs.wait_stream(stream)
        torch.cuda.synchronize()
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg, stream=gs):
            plan.txv(Hs[0], Xs[0], Ys[0], None, gs)
        for _ in range(3):
            cg.replay()
        torch.cuda.synchronize()
        ga, gb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ga.record(stream)
        for _ in range(args.steps):
            cg.replay()
        gb.record(stream)
        torch.cuda.synchronize()
        local_gms = ga.elapsed_time(gb) / args.steps
        del cg
    except Exception as exc:  # report, do not fail the benchmark
        graph = {"error": str(exc)[:200]}
    # every rank takes part in the max, whether or not its capture worked
    gms = max_over_ranks(local_gms, dist, dev)
    if graph is None:
        if gms != float("inf"):  # every rank timed its replays
            graph = {"value": aggregate_rate(world, len(batch), gms / 1000.0), "unit": "products/s",
                     "ms_per_step": gms, "note": "replays of one captured step on one input copy (L2-warm)"}
        else:
            graph = {"error": "graph replay failed on another rank"}

    # end to end through the host-buffer entry point
    hh = torch.tensor(batch.h, dtype=torch.float32).pin_memory()
    xh = torch.tensor(batch.x, dtype=torch.float32).pin_memory()
    yh = torch.zeros(batch.y_len, dtype=torch.float32).pin_memory()
    for _ in range(2):
        plan.txv_host(hh, xh, yh, None, stream)
    e2e_steps = max(3, args.steps // 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        plan.txv_host(hh, xh, yh, None, stream)
    e2e_dt = max_over_ranks((time.perf_counter() - t0) / e2e_steps, dist, dev)
    e2e = {"value": aggregate_rate(world, len(batch), e2e_dt), "unit": "products/s",
           "h2d_bytes_per_step": int(hh.numel() * 4 + xh.numel() * 4), "d2h_bytes_per_step": int(yh.numel() * 4),
           "ms_per_step": 1000.0 * e2e_dt}

    # plain FP64 path: one tensor per launch, same tensors
    fp64 = None
    if not args.no_fp64 and rank == 0:
        p64 = hk.Plan(descs, hk.R64, hk.SAME_X | hk.ONE_PER_LAUNCH)
        H64 = torch.tensor(batch.h, dtype=torch.float64, device=dev)
        X64 = torch.tensor(batch.x, dtype=torch.float64, device=dev)
        Y64 = torch.zeros(batch.y_len, dtype=torch.float64, device=dev)
        p64.txv(H64, X64, Y64, None, stream)
        torch.cuda.synchronize()
        reps = 2
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            p64.txv(H64, X64, Y64, None, stream)
        b.record(stream)
        torch.cuda.synchronize()
        ms64 = a.elapsed_time(b) / reps
        # agreement of the two paths on the same tensors (per-tensor relative inf-norm)
        y32 = Ys[(args.warmup + args.steps - 1) % copies].double().cpu().numpy()
        y64 = Y64.cpu().numpy()
        worst = 0.0
        for i in range(len(batch)):
            o, n = batch.y_off[i], batch.dims[i]
            r = y64[o:o + n]
            worst = max(worst, float(np.max(np.abs(y32[o:o + n] - r)) / np.max(np.abs(r))))
        fp64 = {"value": len(batch) / (ms64 / 1000.0), "unit": "products/s", "ms_per_step": ms64,
                "launches_per_step": int(p64.info["launches"]), "speedup_fp32_batched": (ms64 / ms),
                "fp32_vs_fp64_max_rel_err": worst}
        p64.close()

    secondary = None
    if not args.no_secondary and rank == 0:
        secondary = secondary_workloads(dev, stream)

    cpu, accuracy = None, None
    if pool is not None:
        v, n, dt = cpu_oracle(seconds=15.0, pool=pool, cores=cores)
        cpu = {"value": v, "unit": "products/s", "cores": cores, "kind": "oracle",
               "sample": "first %d tensors of the same 8192-tensor batch, FP64 radix-2 embedding FFT, "
                         "spawn pool of %d processes, %.1f s" % (n, cores, dt)}
        # the timed step's output against the oracle, every tensor
        y_last = Ys[(args.warmup + args.steps - 1) % copies].double().cpu().numpy()
        t0 = time.perf_counter()
        err = oracle_errors(batch, y_last, rank_seed(rank), pool)
        accuracy = {"max_rel_err": float(err.max()), "median_rel_err": float(np.median(err)),
                    "tensors": int(err.size), "norm": "per-tensor relative infinity norm",
                    "against": "FP64 oracle (radix-2 embedding at a power-of-two length)",
                    "oracle_seconds": time.perf_counter() - t0}
        pool.close()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "products/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": bench_config(batch, copies),
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic,
                             "peak_source": peak_src, "kernel": "fast_fwd_kernel<false>",
                             "launches_per_step": int(info["launches"]),
                             "algorithmic_bytes_per_step": alg_bytes},
                "roofline_alu": alu_roofline(alg_flops, kernel_ms, clocks,
                                             torch.cuda.get_device_properties(dev).multi_processor_count),
                "accuracy": accuracy,
                "e2e": e2e, "gpu_launches": int(info["launches"]) * args.steps,
                "plan": info, "tuning": tuning, "fp64_plain": fp64, "cpu_baseline": cpu, "clocks": clocks,
                "secondary": secondary, "graph_replay": graph,
                "step_ms_min": float(np.min(step_ms)), "step_ms_median": float(np.median(step_ms))}
        print(json.dumps(line))
    plan.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
