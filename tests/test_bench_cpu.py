"""Host-side pieces of bench.py on CPU: the clock log it reads back, the
FP32 ALU roofline arithmetic, the peak it divides by, and the traffic record
it reports (a number only while the kernel sources are those it was taken on)."""

import json
import os
import shutil

import pytest

import bench


class _Done:
    """Stands in for the nvidia-smi sampler process (already finished)."""

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _log(tmp_path, rows):
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(", ".join(r) for r in rows) + "\n")
    return str(p)


def test_read_clocks_median_max_and_reasons(tmp_path):
    rows = [
        # index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
        ["0", "2070", "2070", "900.1", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["0", "1965", "2070", "1390.0", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
        ["0", "2070", "2070", "1200.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["1", "300", "2070", "90.0", "0x0", "Active", "Not Active", "Not Active", "Not Active"],  # other GPU
        ["0", "[N/A]", "2070", "0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],  # unparsable
    ]
    c = bench.read_clocks(_log(tmp_path, rows), _Done(), 0)
    assert c["samples"] == 3
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]  # the other GPU's hw_slowdown is not this run's
    assert "soak" in c["window"]


def test_read_clocks_without_sampler_or_samples(tmp_path):
    assert bench.read_clocks(str(tmp_path / "missing.csv"), None, 0) is None
    assert bench.read_clocks(_log(tmp_path, [["1", "2070", "2070", "1", "0", "a", "b", "c", "d"]]), _Done(), 0) is None


def test_alu_roofline_arithmetic():
    r = bench.alu_roofline(flops=1.0e9, kernel_ms=0.5, clocks={"sm_mhz": 2000.0}, sms=152)
    peak = 2 * 128 * 152 * 2000e6 / 1e12  # FMA lanes x SMs x clock, TFLOP/s
    assert r["peak"] == pytest.approx(peak)
    assert r["achieved"] == pytest.approx(2.0)  # 1 GFLOP in 0.5 ms
    assert r["frac"] == pytest.approx(2.0 / peak)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert "152 SMs" in r["peak_source"]
    # no clock record: the maximum SM clock
    assert bench.alu_roofline(1.0e9, 0.5, None, 152)["peak"] == pytest.approx(2 * 128 * 152 * 2070e6 / 1e12)
    # the SM count is the device's, not a constant
    r = bench.alu_roofline(1.0e9, 0.5, {"sm_mhz": 2000.0}, sms=148)
    assert r["peak"] == pytest.approx(2 * 128 * 148 * 2000e6 / 1e12) and "148 SMs" in r["peak_source"]


def test_peak_is_the_measured_copy_bandwidth():
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if not os.path.exists(path):  # written per machine, not part of the sources
        assert bench.peaks() == (6800.0, "fallback")
        return
    with open(path) as f:
        measured = float(json.load(f)["hbm_gbs"])
    assert bench.peaks() == (measured, "measured")


def test_traffic_record_follows_the_sources(tmp_path, monkeypatch):
    import hashlib
    # a tree with two kernel sources and a record taken on them
    root = tmp_path / "tree"
    srcs = ["pkg/a.cu", "pkg/b.cuh"]
    for rel, text in zip(srcs, ["// kernel\n", "// header\n"]):
        (root / rel).parent.mkdir(parents=True, exist_ok=True)
        (root / rel).write_text(text)
    h = hashlib.sha256()
    for rel in srcs:
        h.update((root / rel).read_bytes())
    (root / "profiles").mkdir()
    rec = {"bytes_per_step": 123456, "sources": srcs, "sources_sha256": h.hexdigest()}
    (root / "profiles" / "fast_fwd_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.profiled_traffic() == 123456
    with open(root / srcs[1], "a") as f:
        f.write("// changed\n")
    assert bench.profiled_traffic() is None
    # no record at all
    os.remove(root / "profiles" / "fast_fwd_traffic.json")
    assert bench.profiled_traffic() is None


def test_both_arms_print_one_config():
    from paper_1401_6238_gb300 import workloads as wl
    b = wl.batched_square(count=8192, seed=bench.rank_seed(0))
    a, c = bench.bench_config(b, 6), bench.bench_config(wl.batched_square(count=8192, seed=bench.rank_seed(0)), 6)
    assert a == c
    assert "FP32" not in a["workload"] and "f64" not in json.dumps(a)  # dtype carries the precision


class _SerialPool:
    def map(self, fn, tasks):
        return [fn(t) for t in tasks]


def test_oracle_errors_over_a_batch():
    import numpy as np
    import oracle
    from paper_1401_6238_gb300 import workloads as wl
    full = wl.batched_square(count=8192, seed=1)
    b = full.subset(np.arange(70))
    y = np.zeros(b.y_len)
    for i in range(len(b)):
        m, n, h, x = b.tensor(i)
        y[b.y_off[i]: b.y_off[i] + n] = oracle.fast_y(h, [x] * (m - 1), [n] * m).real
    assert np.all(bench.oracle_errors(b, y, 1, _SerialPool()) == 0.0)
    # a relative error planted in tensor 37 is reported there alone
    o, n = b.y_off[37], b.dims[37]
    y[o + n // 2] += 1e-4 * np.max(np.abs(y[o:o + n]))
    e = bench.oracle_errors(b, y, 1, _SerialPool())
    assert e[37] == pytest.approx(1e-4) and np.all(np.delete(e, 37) == 0.0)


def test_autotune_fp64_threshold_rule():
    from paper_1401_6238_gb300 import autotune as at
    # FP64 powers that never help: never chosen
    e32 = {m: 3e-6 * m for m in range(2, 9)}
    assert at.fp64_threshold(e32, dict(e32)) == 99
    # they pay from m = 6 up (error cut in half, FP32 error above half the bound)
    e32 = {2: 1e-6, 3: 1e-6, 4: 2e-6, 5: 4e-6, 6: 6e-6, 7: 8e-6, 8: 9e-6}
    e64 = {m: (v / 2 if m >= 6 else v) for m, v in e32.items()}
    assert at.fp64_threshold(e32, e64) == 6
    # a gain below the bound's half does not count, nor a gap at the top
    e64 = {m: v / 2 for m, v in e32.items()}
    assert at.fp64_threshold(e32, e64) == 6
    e64[8] = e32[8]
    assert at.fp64_threshold(e32, e64) == 99


def test_autotune_bin_batches_fall_in_their_bins():
    from paper_1401_6238_gb300 import autotune as at
    for i, L in enumerate(at.BINS):
        lo = at.BINS[i - 1] if i else 0
        b = at.bin_batch(L, (3, 4, 5), 16, seed=L) or at.bin_batch(L, (2,), 16, seed=L)
        d = b.orders * (b.dims - 1) + 1
        assert len(b) == 16 and (d > lo).all() and (d <= L).all()
