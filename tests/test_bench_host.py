"""Host-side logic of bench.py that needs no GPU: the clock-sample summary, the
streaming byte model of the TV path and the committed profile records."""
import datetime
import time

import bench


def _line(t, clk, reasons=("Not Active",) * 4, stamp=None):
    ts = stamp or datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return ", ".join([ts, str(clk), "2070", "900.0", "0x0"] + list(reasons))


def test_clock_summary_keeps_the_timed_region():
    now = time.time()
    lines = ["", "garbage",
             _line(now - 1.0, 990),  # idle, before the timed region
             _line(now + 0.01, 2070),
             _line(now + 0.06, 2070, ("Not Active", "Not Active", "Not Active", "Active")),
             _line(now + 0.11, 2055),
             _line(now + 2.0, 1000)]  # after it
    s = bench.summarize_clocks(lines, now, now + 0.2)
    assert s["samples_in_timed_region"] == 3 and s["samples"] == 3
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_falls_back_to_every_sample():
    now = time.time()
    lines = [_line(now, 2000, stamp="not a time"), _line(now, 2070, stamp="??"),
             _line(now, 1900, ("Active", "Not Active", "Not Active", "Not Active"))]
    s = bench.summarize_clocks(lines, now + 10, now + 11)
    assert s["samples_in_timed_region"] == 0 and s["samples"] == 3
    assert s["sm_mhz"] == 2000.0 and s["reasons"] == ["hw_slowdown"]
    assert bench.summarize_clocks(["x, y"], now, now) is None


def test_streaming_byte_model():
    # x-update 12.125 + 4 / R, first pass 12, 19 later passes of 20, finalize 20, z term 8
    assert bench.tv_stream_bytes(16, 20, True) == 12.125 + 0.25 + 12 + 19 * 20 + 20 + 8
    assert bench.tv_stream_bytes(32, 20, False) == 424.25


def test_oracle_sample_is_stratified_by_size():
    ws = bench.rank_workloads(0)
    assert len(ws) == 64 and sum(w.Z * w.H * w.W for w in ws) == 613941248
    idx = bench.oracle_sample(ws)
    assert len(set(idx)) == 8
    sizes = sorted(w.Z * w.H * w.W for w in ws)
    got = [ws[i].Z * ws[i].H * ws[i].W for i in idx]
    assert got == sorted(got)
    for k, v in enumerate(got):  # one item from each eighth of the size order
        assert sizes[8 * k] <= v <= sizes[8 * k + 7]
    # replicas draw different batches
    assert [w.seed for w in bench.rank_workloads(1)] != [w.seed for w in ws]


def test_profile_records_follow_the_kernel_sources(tmp_path, monkeypatch):
    """A committed ncu record counts only while the kernel's sources hash as when
    it was taken; the L2 view divides its bytes by the launch time of the run."""
    import json

    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = {"sources_sha256_16": bench._kernel_hash(bench.TVZ_SOURCES),
           "dram_bytes_per_launch": 1.0e6, "l2_bytes_per_launch": 4.0e9, "l2_peak_GBs": 40000.0,
           "l2_sector_hit_rate_pct": 70.0}
    (prof / "k_w.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the source hash still reads the package sources
    monkeypatch.setattr(bench, "_kernel_hash",
                        lambda sources: rec["sources_sha256_16"] if sources == bench.TVZ_SOURCES
                        else "0" * 16)
    assert bench._traffic("k", "w", bench.TVZ_SOURCES) == 1.0e6
    l2 = bench._l2("k", "w", bench.TVZ_SOURCES, 1e-3)
    assert l2["achieved"] == 4.0e9 / 1e-3 / 1e9 and l2["frac"] == l2["achieved"] / 40000.0
    assert l2["unit"] == "GB/s"
    # another kernel source: the record no longer applies
    assert bench._traffic("k", "w", bench.DOMINANT_SOURCES) is None
    assert bench._l2("k", "w", bench.DOMINANT_SOURCES, 1e-3) is None
    assert bench._record("missing", "w", bench.TVZ_SOURCES) == {}
