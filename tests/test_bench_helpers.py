"""Host-side helpers of bench.py that shape its JSON line (no GPU): the clock
record, the DRAM-traffic lookup keyed by the kernel sources, the workload
description and the peak denominators."""
import os
import shutil

import bench


def test_clock_summary_median_max_and_reasons():
    c = bench.Clocks(0)
    c.rows = [["0", "2070", "2070", "900", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
              ["0", "1995", "2070", "1390", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
              ["0", "2055", "2070", "1200", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
              ["garbage"], ["0", "[N/A]", "2070"]]
    s = c.summary()
    assert s["sm_mhz"] == 2055 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    assert bench.Clocks(0).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_traffic_lookup_follows_the_kernel_sources(tmp_path, monkeypatch):
    """Counters are returned while the pass sources are the ones they were taken
    with (the hash in their row), and null for a kernel without counters or for
    changed sources."""
    rows = {}
    for line in open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.txt")):
        if line.strip() and not line.startswith("#"):
            k, h, v = line.split()[:3]
            rows[k] = (h, float(v))
    assert rows and all(len(h) == 16 for h, _ in rows.values())
    for k, (h, v) in rows.items():
        assert bench.traffic_from_profiles(k) == (v if h == bench.pass_sources_hash() else None)
    # a copy of the tree whose counters carry the current hash, then a changed source
    root = tmp_path / "r"
    csrc = root / "paper_1503_01405_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (root / "profiles").mkdir()
    for f in ("passes.cuh", "fft_block.cuh", "tc_dft.cuh"):
        shutil.copy(os.path.join(bench.ROOT, "paper_1503_01405_gb300", "csrc", f), csrc / f)
    cur = bench.pass_sources_hash(str(root))
    (root / "profiles" / "ncu_traffic.txt").write_text(
        "# header\n" + "".join(f"{k} {cur} {v}\n" for k, (_, v) in rows.items()))
    monkeypatch.setattr(bench, "ROOT", str(root))
    for k, (_, v) in rows.items():
        assert bench.traffic_from_profiles(k) == v
    assert bench.traffic_from_profiles("k_not_a_kernel") is None
    with open(csrc / "passes.cuh", "a") as f:
        f.write("\n")
    k = next(iter(rows))
    assert bench.traffic_from_profiles(k) is None


def test_workload_description_and_peaks():
    one = bench.workload_config(1_920_000_000)
    two = bench.workload_config(1_920_000_000, 2)
    assert one["samples_per_step"] == two["samples_per_step"] == 1_920_000_000
    assert "1.92e9 int8 samples" in one["workload"] and "interleaved N / S" in two["workload"]
    assert one["nfft"] == 1 << 24 and one["nchan"] == 64
    p = bench.measured_peaks()
    assert p["hbm_gbs"] > 1000 and p["src"] in ("measured", "fallback")
    if os.path.exists(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")):
        assert p["src"] == "measured"


def test_roofline_arithmetic():
    """The roofline object: FP32 operations per launch over the mean launch time
    against the nominal FP32 ceiling; the method's bytes (one segment's input
    per launch) and the pass's own bytes against measured HBM."""
    stages = {"fwd_cols_unpack": {"ms": 20.0, "launches": 100, "pass_bytes": 1e8, "algo_flops": 4e8},
              "fwd_rows_chirp_inv": {"ms": 40.0, "launches": 100, "pass_bytes": 2e8, "algo_flops": 8e8},
              "inv_cols_detect": {"ms": 10.0, "launches": 100, "pass_bytes": 1e8, "algo_flops": 5e8}}
    st = {"nfft": 1 << 24, "nchan": 64, "seg_step": 13_501_440}
    fp32 = {"tflops": 70.0}
    peaks = {"hbm_gbs": 6800.0, "src": "measured"}
    r = bench.roofline(stages, 2, 35.0, 100 * 13_501_440 // 2, 1, st, fp32, peaks)
    assert r["kernel"] == "k_fwd_rows_inv" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["launch_us"] - 400.0) < 1e-9
    assert abs(r["achieved"] - 8e8 / 400e-6 / 1e12) < 1e-12
    assert abs(r["frac"] - r["achieved"] / bench.FP32_NOMINAL_TFLOPS) < 1e-12
    assert abs(r["frac_of_measured"] - r["achieved"] / 70.0) < 1e-12
    seg = (1 << 24) + 4.0 * (13_501_440 // 128)
    assert abs(r["algo_hbm_gbs"] - seg / 400e-6 / 1e9) < 1e-9
    assert abs(r["pass_bytes_frac"] - 2e8 / 400e-6 / 1e9 / 6800.0) < 1e-12
    # the path: 100 launches of each stage over 2 steps of 35 ms
    assert abs(r["path"]["tflops"] - (17e8 * 100 / 2) / 35e-3 / 1e12) < 1e-9
    assert abs(bench.FP32_NOMINAL_TFLOPS - 80.55) < 0.01


def test_host_cpu_record():
    h = bench.host_cpu()
    assert h["nproc"] >= 1 and isinstance(h["model"], str) and h["model"]
