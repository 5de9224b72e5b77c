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
    r = bench.alu_roofline(flops=1.0e9, kernel_ms=0.5, clocks={"sm_mhz": 2000.0})
    peak = 2 * 128 * 152 * 2000e6 / 1e12  # FMA lanes x SMs x clock, TFLOP/s
    assert r["peak"] == pytest.approx(peak)
    assert r["achieved"] == pytest.approx(2.0)  # 1 GFLOP in 0.5 ms
    assert r["frac"] == pytest.approx(2.0 / peak)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    # no clock record: the maximum SM clock
    assert bench.alu_roofline(1.0e9, 0.5, None)["peak"] == pytest.approx(2 * 128 * 152 * 2070e6 / 1e12)


def test_peak_is_the_measured_copy_bandwidth():
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if not os.path.exists(path):  # written per machine, not part of the sources
        assert bench.peaks() == (6800.0, "fallback")
        return
    with open(path) as f:
        measured = float(json.load(f)["hbm_gbs"])
    assert bench.peaks() == (measured, "measured")


def test_traffic_record_follows_the_sources(tmp_path, monkeypatch):
    rec_path = os.path.join(bench.ROOT, "profiles", "real_fwd_traffic.json")
    with open(rec_path) as f:
        rec = json.load(f)
    # a copy of the tree holding the recorded sources, one of them changed
    root = tmp_path / "tree"
    for rel in rec["sources"] + ["profiles/real_fwd_traffic.json"]:
        dst = root / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, rel), dst)
    monkeypatch.setattr(bench, "ROOT", str(root))
    same = bench.profiled_traffic()
    with open(root / rec["sources"][0], "a") as f:
        f.write("\n// changed\n")
    assert bench.profiled_traffic() is None
    # the unchanged copy reports the recorded bytes when the record matches it
    if same is not None:
        assert same == rec["bytes_per_step"]
