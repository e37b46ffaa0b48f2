"""The benchmark's roofline traffic comes from the committed record of an ncu
capture of the colour pass, and only while the kernel sources are the ones
that were profiled."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _write(path, tpu, sha):
    with open(path, "w") as f:
        json.dump({"dram_bytes_per_gap_update": tpu, "kernel_sources_sha16": sha}, f)


def test_record_is_read_for_its_kernel_sources(monkeypatch, tmp_path):
    rec = tmp_path / "traffic.json"
    _write(rec, 12.5, bench.kernel_sources_hash())
    monkeypatch.setattr(bench, "TRAFFIC_RECORD", str(rec))
    assert bench.recorded_traffic_per_update() == 12.5


def test_record_is_ignored_when_the_sources_change(monkeypatch, tmp_path):
    rec = tmp_path / "traffic.json"
    _write(rec, 12.5, "0" * 16)
    monkeypatch.setattr(bench, "TRAFFIC_RECORD", str(rec))
    assert bench.recorded_traffic_per_update() is None


def test_record_is_ignored_without_a_record(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "TRAFFIC_RECORD", str(tmp_path / "missing.json"))
    assert bench.recorded_traffic_per_update() is None


def test_committed_record_when_present_is_plausible():
    if not os.path.exists(bench.TRAFFIC_RECORD):
        return
    with open(bench.TRAFFIC_RECORD) as f:
        rec = json.load(f)
    # DRAM bytes per gap site-update: below the 14 B algorithmic figure plus the
    # realisation sums' share, and far above zero
    assert 6.0 < float(rec["dram_bytes_per_gap_update"]) < 20.0
    assert len(rec["kernel_sources_sha16"]) == 16


def test_record_is_written_from_an_ncu_raw_page(monkeypatch, tmp_path):
    """`bench.py --record-traffic` takes the DRAM bytes of the sampling launch (the
    colour pass whose accumulation argument is 1) from `ncu --page raw --csv` output
    and divides by the gap site-updates of one launch on the field of that side."""
    import csv
    import synthetic
    raw = tmp_path / "raw.csv"
    with open(raw, "w", newline="") as f:
        w = csv.writer(f)
        w.writerow(["ID", "Kernel Name", "dram__bytes_read.sum", "dram__bytes_write.sum"])
        w.writerow(["", "", "Mbyte", "Kbyte"])
        w.writerow(["0", "void tiled_pass_kernel<16, 16, 4, 16, 0, 0>(SweepArgs)", "9.0", "9.0"])
        w.writerow(["1", "void tiled_pass_kernel<16, 16, 4, 16, 1, 0>(SweepArgs)", "2.0", "500.0"])
    rec = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "TRAFFIC_RECORD", str(rec))
    bench.record_traffic(str(raw), 64, "ncu ...")
    wl = synthetic.workload("lognormal4096", L=64)
    updates = int(wl.gap[0].sum()) * wl.chains / 2.0
    with open(rec) as f:
        got = json.load(f)
    assert got["dram_bytes_per_gap_update"] == round(2.5e6 / updates, 4)
    assert got["kernel_sources_sha16"] == bench.kernel_sources_hash()
    assert bench.recorded_traffic_per_update() == got["dram_bytes_per_gap_update"]
