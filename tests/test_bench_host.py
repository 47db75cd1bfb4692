"""Host-side logic of bench.py: the accuracy metrics of the h_max sweep (the paper's
"aligned" = confidently mapped reads, "errors" = confident reads at the wrong place)."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
import synth  # noqa: E402

RESULT = np.dtype([("location", "<i8"), ("edit_distance", "<i4"), ("strand", "u1"),
                   ("cls", "u1"), ("pad", "u1", 2)])


def _reads(origin, strand):
    n = len(origin)
    return synth.Reads(np.zeros(0, np.uint8), np.zeros(n + 1, np.uint64),
                       np.asarray(origin, np.int64), np.asarray(strand, np.uint8),
                       np.zeros(n, np.uint32))


def test_accuracy_counts_each_case():
    rd = _reads([1000, 2000, 3000, 4000, 5000, 6000], [0, 1, 0, 1, 0, 0])
    got = np.zeros(6, RESULT)
    # 0: single, exact; 1: single, 20 bases off (still correct); 2: single, 21 off (wrong)
    # 3: single, wrong strand; 4: multiple; 5: not found
    got["cls"] = [1, 1, 1, 1, 2, 0]
    got["location"] = [1000, 2020, 3021, 4000, 5000, -1]
    got["strand"] = [0, 1, 0, 0, 0, 0]
    a = bench.accuracy(got, rd)
    assert np.isclose(a["aligned_pct"], 100.0 * 4 / 6)
    assert np.isclose(a["error_pct"], 100.0 * 2 / 4)
    assert np.isclose(a["multiple_pct"], 100.0 / 6) and np.isclose(a["not_found_pct"], 100.0 / 6)


def test_accuracy_with_no_confident_reads():
    rd = _reads([10, 20], [0, 0])
    got = np.zeros(2, RESULT)
    got["cls"] = [0, 2]
    a = bench.accuracy(got, rd)
    assert a["aligned_pct"] == 0.0 and a["error_pct"] == 0.0


def test_cpu_oracle_sample_reports_all_cores_and_one_core():
    # the bench's CPU baseline: the oracle as it stands, timed on a bounded sample on
    # all host cores and on one; the sample's results are the oracle's own
    import oracle
    w = synth.CONFIGS["C1"].scaled(G=300_000, n_reads=3000)
    g, _ = w.make_genome()
    rd = w.make_reads(g)
    cb, sample, res = bench.cpu_oracle_sample(w, g, rd, None, target_s=0.2)
    assert cb["kind"] == "oracle" and cb["cores"] == (os.cpu_count() or 1)
    assert cb["value"] > 0 and cb["single_core"]["value"] > 0
    assert 200 <= cb["single_core"]["reads"] <= len(sample)
    ref, _ = oracle.Index(g, w.seed_len).align(rd.bases, rd.offsets, **w.params())
    for f in ("location", "edit_distance", "strand", "cls"):
        assert np.array_equal(res[f], ref[f][:len(sample)])
