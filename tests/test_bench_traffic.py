"""The benchmark's roofline traffic comes from the committed ncu summary of the
colour pass, and only while the kernel sources are the ones that were profiled."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_committed_record_is_read_for_its_kernel_sources(monkeypatch):
    import re
    with open(bench.TRAFFIC_PROFILE) as f:
        m = re.search(r"traffic record: ([0-9.]+) B per gap site-update, kernel sources ([0-9a-f]+)",
                      f.read())
    assert m, "no traffic record line in the colour-pass summary"
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda: m.group(2))
    tpu = bench.recorded_traffic_per_update()
    # DRAM bytes per gap site-update: below the 14 B algorithmic figure plus the
    # realisation sums' share, and far above zero
    assert tpu == float(m.group(1)) and 8.0 < tpu < 16.0


def test_record_is_ignored_when_the_sources_change(monkeypatch):
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda: "0" * 16)
    assert bench.recorded_traffic_per_update() is None


def test_record_is_ignored_without_a_summary(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(tmp_path / "missing.md"))
    assert bench.recorded_traffic_per_update() is None
