"""Host-side logic of bench.py that needs no GPU: the rule that a recorded DRAM-traffic ratio is used
only while the Wilson kernel's source is the one it was measured on, and the measured-peak lookup."""
from __future__ import annotations

import json

import bench


def test_traffic_ratios_follow_the_kernel_source(monkeypatch):
    monkeypatch.setattr(bench, "KERNEL_SHA", bench.kernel_sha())  # as if measured on this source
    for key, ratio in bench.DRAM_OVER_ALGORITHMIC.items():
        assert bench.dram_ratio(key) == ratio
        assert 0.0 < ratio <= 1.2
    assert bench.dram_ratio("f32_no_such_case") is None
    monkeypatch.setattr(bench, "KERNEL_SHA", "0" * 16)
    for key in bench.DRAM_OVER_ALGORITHMIC:
        assert bench.dram_ratio(key) is None


def test_measured_peaks_are_read_from_the_driver_file():
    with open(bench.os.path.join(bench.ROOT, "MEASURED_PEAKS.json")) as fh:
        raw = json.load(fh)
    assert bench.measured_peaks() == (float(raw["hbm_gbs"]), "measured")
