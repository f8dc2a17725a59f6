"""Host-side logic of bench.py (no GPU): the ncu traffic records the bench line
quotes, and the §3.5 per-read locus statistics of the threshold regime."""
import json
import os

import numpy as np

import bench


def test_traffic_records_are_consistent():
    """Each committed traffic record scales its capture's DRAM bytes by its
    stated factor, and a record is only quoted for the launch it was scaled to
    (the batch) and for the kernel source it was taken on."""
    for workload, (name, kernel, batch) in bench.TRAFFIC_RECORDS.items():
        path = os.path.join(bench.ROOT, "profiles", name)
        assert os.path.exists(path), path
        rec = json.load(open(path))
        assert rec["capture"].startswith("profiles/") and os.path.exists(os.path.join(bench.ROOT, rec["capture"]))
        per = rec["dram_bytes_read"] + rec["dram_bytes_write"]
        assert abs(rec["dram_bytes_per_launch"] - per) <= 1e-9 * per
        assert abs(rec["dram_bytes_per_launch_scaled"] - per * rec["scale_factor"]) <= 1e-9 * per * rec["scale_factor"]
        assert len(rec["kernel_sha"]) == 16
        assert bench.traffic_record(workload, batch + 1) is None  # another launch: not quoted
        got = bench.traffic_record(workload, batch)
        assert got is None or got["kernel_sha"] == rec["kernel_sha"]
    assert bench.traffic_record("no_such_workload", 1) is None


def test_locus_stats():
    """Three reads, window step 10, window length 100: read 0 has one run of
    overlapping windows at its planted start (one locus, found); read 1 has
    two runs far apart, neither near its start (two loci, missed); read 2 has
    no output at all (no locus, missed)."""
    reads = np.array([0, 0, 0, 1, 1, 1], dtype=np.int64)
    wins = np.array([50, 52, 55, 10, 11, 500], dtype=np.int64)  # window numbers
    true_pos = np.array([510, 2000, 300], dtype=np.int64)
    st = bench.locus_stats(reads, wins, true_pos, 3, stride=10, N=100)
    assert st["loci_per_read"] == (1 + 2 + 0) / 3
    assert st["unique_fraction"] == 1 / 3
    assert st["missed_fraction"] == 2 / 3
    assert st["pairs_per_read"] == 6 / 3
    assert st["reads_without_output"] == 1 / 3
    # the order of the pairs does not matter
    perm = np.array([5, 2, 0, 4, 1, 3])
    assert bench.locus_stats(reads[perm], wins[perm], true_pos, 3, stride=10, N=100) == st
    # no pairs at all
    empty = bench.locus_stats(np.zeros(0, np.int64), np.zeros(0, np.int64), true_pos, 3, stride=10, N=100)
    assert empty["loci_per_read"] == 0 and empty["missed_fraction"] == 1.0


def test_measured_peaks_have_the_roofline_keys():
    peaks, src = bench.measured_peaks()
    assert src in ("measured", "fallback")
    for key in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained"):
        assert peaks[key] > 0
