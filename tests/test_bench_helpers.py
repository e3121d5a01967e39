"""Host logic of bench.py that needs no GPU: the source fingerprint that
decides whether recorded DRAM counters still describe the kernels, the
lookup of those counters, and the peak-bandwidth fallback."""
import json
import os

import bench


def _tree(tmp_path, files):
    d = tmp_path / "paper_2209_15040_gb300" / "csrc"
    d.mkdir(parents=True, exist_ok=True)
    for name, text in files.items():
        (d / name).write_text(text)
    return tmp_path


def test_fingerprint_follows_kernel_sources(tmp_path, monkeypatch):
    root = _tree(tmp_path, {"pass_kernels.cuh": "x", "pass_c32.cu": "y", "wsfft_api.cu": "z",
                            "transpose.cu": "other kernel", "notes.txt": "ignored"})
    monkeypatch.setattr(bench, "ROOT", str(root))
    csrc = root / "paper_2209_15040_gb300" / "csrc"
    h0 = bench.source_sha256()
    (csrc / "notes.txt").write_text("changed")
    (csrc / "transpose.cu").write_text("changed")
    assert bench.source_sha256() == h0  # files outside the benchmark plan's kernels do not count
    (csrc / "pass_c32.cu").write_text("y2")
    assert bench.source_sha256() != h0
    (csrc / "pass_c32.cu").write_text("y")
    assert bench.source_sha256() == h0
    (csrc / "fft_core.cuh").write_text("")
    assert bench.source_sha256() != h0  # a listed file that appears counts too


def test_traffic_lookup_only_for_matching_sources(tmp_path, monkeypatch):
    root = _tree(tmp_path, {"pass_kernels.cuh": "kernel"})
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.kernel_traffic(0) is None  # no record
    (root / "profiles").mkdir()
    rec = {"source_sha256": bench.source_sha256(), "c32_512_pass0": 1.5e9, "c32_512_pass2": 2.0e9}
    (root / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.kernel_traffic(0) == 1.5e9
    assert bench.kernel_traffic(2) == 2.0e9
    assert bench.kernel_traffic(1) is None  # not recorded
    (root / "paper_2209_15040_gb300" / "csrc" / "pass_kernels.cuh").write_text("kernel, edited")
    assert bench.kernel_traffic(0) is None  # counters of older kernels are not reported


def test_recorded_traffic_is_a_plausible_launch():
    # the committed record, when it matches the sources, holds about one read
    # and one write of the 1 GiB array per launch (not a multiple of it)
    path = os.path.join(bench.ROOT, "profiles", "traffic.json")
    with open(path) as f:
        rec = json.load(f)
    for i in range(3):
        v = rec.get("c32_512_pass%d" % i)
        assert v is None or 0.9 * 2 ** 31 < v < 1.2 * 2 ** 31, (i, v)


def test_peak_fallback_without_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6791.0}))
    assert bench.peaks() == (6791.0, "measured")


def test_device_info_is_safe_without_a_gpu():
    import torch
    info = bench.device_info(torch.device("cuda", 0))
    assert info is None or (isinstance(info["name"], str) and info["sms"] > 0)


def test_clock_samples_filtered_to_the_timed_region():
    from datetime import datetime
    import bench

    def line(ts, mhz, reason="Not Active"):
        stamp = datetime.fromtimestamp(ts).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return f"{stamp}, {mhz}, 2070, 500.0, {reason}, Not Active, Not Active, Not Active"

    t0 = 1_800_000_000.0
    lines = [line(t0 - 1.0, 900, "Active"), line(t0 + 0.02, 2070), line(t0 + 0.03, 2060), line(t0 + 2.0, 1000)]
    out = bench.Clocks.parse(lines, (t0, t0 + 0.04))
    assert out["samples_in_timed_region"] == 2 and out["sm_mhz"] == 2065 and out["reasons"] == []
    out = bench.Clocks.parse(lines, (t0 + 5, t0 + 6))  # nothing inside: every sample counts
    assert out["samples_in_timed_region"] == 0 and out["samples"] == 4 and out["reasons"] == ["hw_slowdown"]
