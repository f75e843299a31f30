"""bench.py's ncu side record (CPU only).

record_ncu turns the raw page of one capture per sweep kernel into the
record the roofline fields read: DRAM bytes (read + write) and warp
instructions per stage, the captured durations, and the hash of the kernel
sources, so that a record of other kernels is recognised as stale.  A Potts
sweep has no bond kernel (its labeling kernel draws the bonds), so that
stage may be missing; the three others may not.
"""
import csv
import json

import pytest

import bench

HEADER = ["ID", "Kernel Name", "dram__bytes_read.sum", "dram__bytes_write.sum", "smsp__inst_executed.sum",
          "gpu__time_duration.sum"]
UNITS = ["", "", "Mbyte", "Kbyte", "inst", "usecond"]


def write_csv(path, rows):
    with open(path, "w", newline="") as f:
        w = csv.writer(f)
        w.writerow(HEADER)
        w.writerow(UNITS)
        for r in rows:
            w.writerow(r)


def test_record_reads_bytes_instructions_and_durations(tmp_path):
    src = tmp_path / "raw.csv"
    out = tmp_path / "traffic.json"
    write_csv(src, [
        ["0", "void (anonymous namespace)::k_label_tiles<true, false, true>(swgb::Batch)", "16.8", "750", "83,600,000",
         "119.5"],
        ["1", "void (anonymous namespace)::k_merge<false>(swgb::Batch)", "5.25", "5", "5,000,000", "20.8"],
        ["2", "void (anonymous namespace)::k_flip_tiles<true, false, false, false>(swgb::Batch)", "36", "80",
         "11,500,000", "25.1"],
        # A second launch of a stage is ignored: the first capture counts.
        ["3", "void (anonymous namespace)::k_merge<false>(swgb::Batch)", "99", "99", "1", "1"],
    ])
    rec = bench.record_ncu(str(src), "test capture", out=str(out))
    assert json.load(open(out)) == rec
    assert rec["source"] == "test capture"
    assert rec["kernel_source_sha256"] == bench.kernel_source_sha256()
    assert rec["label"] == pytest.approx(16.8e6 + 750e3)
    assert rec["merge"] == pytest.approx(5.25e6 + 5e3)
    assert rec["flip"] == pytest.approx(36e6 + 80e3)
    assert rec["warp_instructions"] == {"label": 83.6e6, "merge": 5e6, "flip": 11.5e6}
    assert rec["duration_us"] == {"label": 119.5, "merge": 20.8, "flip": 25.1}
    assert "bonds" not in rec


def test_record_needs_the_labeling_merge_and_flip_kernels(tmp_path):
    src = tmp_path / "raw.csv"
    write_csv(src, [["0", "void (anonymous namespace)::k_merge<false>(swgb::Batch)", "1", "1", "1", "1"]])
    with pytest.raises(SystemExit):
        bench.record_ncu(str(src), "incomplete", out=str(tmp_path / "t.json"))


def test_source_hash_covers_the_kernel_sources():
    h = bench.kernel_source_sha256()
    assert len(h) == 64 and h == bench.kernel_source_sha256()
    assert all(p.endswith((".cu", ".cuh", ".h")) for p in bench.KERNEL_SOURCES)
