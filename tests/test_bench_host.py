"""Host-side logic of bench.py (no GPU): clock sampling summary, roofline arithmetic,
the keying of the committed DRAM-traffic record, the output-site sample and the
reference arm's JSON line."""
import argparse
import json
import os

import numpy as np
import pytest

import bench

NA = "Not Active"


def test_clock_summary_median_and_reasons():
    s = bench.ClockSampler(0)
    s.lines = [
        f"0, 2070, 2070, 900.5, 0x0, {NA}, {NA}, {NA}, {NA}",
        f"0, 1965, 2070, 1390.0, 0x4, {NA}, {NA}, {NA}, Active",
        f"0, 2010, 2070, 1200.0, 0x0, {NA}, {NA}, {NA}, {NA}",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, a, b, c, d",
    ]
    out = bench.ClockSampler.summary(s)
    assert out["sm_mhz"] == 2010.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    s.lines = [f"0, 1500, 2070, 900.0, 0x0, Active, {NA}, Active, {NA}"]
    assert bench.ClockSampler.summary(s)["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    s.lines = []
    assert bench.ClockSampler.summary(s)["reasons"] == ["unsampled"]


def test_compulsory_bytes_follow_the_field_layouts():
    # input-parity spinor + output spinor + 8 links per output site
    spinor = {"f64": 12 * 16, "df64": 12 * 16, "f32": 6 * 16, "f16": 3 * 16 + 4}
    link = {("f64", 18): 9 * 16, ("f64", 12): 6 * 16, ("df64", 18): 9 * 16, ("f32", 18): 72, ("f32", 12): 48,
            ("f16", 18): 36, ("f16", 12): 24}
    for (p, r), b in bench.COMPULSORY.items():
        assert b == 2 * spinor[p] + 8 * link[(p, r)], (p, r)


def test_roofline_entry_arithmetic():
    vh = 1 << 20
    e = bench.roofline_entry(0.125, vh, "f32", 18, 6781.8)
    gbs = 768 * vh / 0.125e-3 / 1e9
    assert e["gbs_compulsory"] == pytest.approx(gbs)
    assert e["frac_of_measured_hbm"] == pytest.approx(gbs / 6781.8)
    assert e["frac_of_8tbs"] == pytest.approx(gbs / 8000.0)
    assert e["gflops"] == pytest.approx(1320 * vh / 0.125e-3 / 1e9)


def test_single_process_aggregate_is_identity():
    assert bench.aggregate_over_ranks(1.5, 10) == (1.5, 10.0)


def test_traffic_record_is_keyed_on_the_kernel_sources(monkeypatch):
    rec_path = os.path.join(bench.ROOT, "profiles", "hop_traffic.json")
    rec = json.load(open(rec_path))
    assert rec["dram_bytes_per_launch"] > 0 and rec["algorithmic_bytes_per_launch"] == 768 * (1 << 20)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: rec["source_sha"])
    assert bench.measured_traffic()[0] == float(rec["dram_bytes_per_launch"])
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.measured_traffic()[0] is None  # stale counters are not reported


def test_output_sites_are_one_parity():
    dims = (4, 2, 4, 6)
    T, Lx, Ly, Lz = dims
    for parity in (0, 1):
        s = bench.output_sites(dims, parity)
        assert len(s) == T * Lx * Ly * Lz // 2 and len(np.unique(s)) == len(s)
        x = s % Lx
        y = (s // Lx) % Ly
        z = (s // (Lx * Ly)) % Lz
        t = s // (Lx * Ly * Lz)
        assert np.all((x + y + z + t) % 2 == parity)


def test_reference_arm_json_line(capsys):
    args = argparse.Namespace(steps=1, warmup=0, gpus=1)
    bench.run_reference(args, 0)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "GFLOP/s"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
