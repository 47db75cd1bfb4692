"""Checks of the seeded input generator against numbers the paper prints.

The "Hash Index" subsection ("Longer Seeds") gives: at a 2% error rate a 20-base
seed is error-free with probability 0.98^20 = 0.67, all five seeds of a 100-base
read carry an error with probability 0.33^5 = 0.004, and a seed of length s matches
about G/4^s locations by chance.  Values are in tests/golden/paper_probabilities.txt.
"""
import os

import numpy as np

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden():
    out = {}
    with open(os.path.join(GOLDEN, "paper_probabilities.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v, tol = line.split()
            out[k] = (float(v), float(tol))
    return out


def _rc(a: bytes) -> bytes:
    return a[::-1].translate(bytes.maketrans(b"ACGT", b"TGCA"))


def test_determinism_and_subranges():
    g1, _ = synth.genome(200_000, 0.05)
    g2, _ = synth.genome(200_000, 0.05, threads=3)
    assert np.array_equal(g1, g2)
    lens = np.full(100, 100, dtype=np.uint32)
    a = synth.reads(g1, lens, 0.01, 0.001, threads=1)
    b = synth.reads(g1, lens[40:], 0.01, 0.001, first_index=40, threads=4)
    assert a.bases[a.offsets[40]:].tobytes() == b.bases.tobytes()
    assert np.array_equal(a.origin[40:], b.origin)
    assert set(np.unique(g1).tolist()) <= set(b"ACGT")


def test_seed_error_probabilities_match_paper():
    gold = _golden()
    g, _ = synth.genome(2_000_000, 0.0)
    n = 200_000
    rd = synth.reads(g, np.full(n, 100, dtype=np.uint32), 0.02, 0.0, seed=123)
    gb = g.tobytes()
    reads = rd.bases.reshape(n, 100)
    ref = np.frombuffer(b"".join(gb[o:o + 100] for o in rd.origin.tolist()), dtype=np.uint8)
    ref = ref.reshape(n, 100)
    fwd = reads.copy()
    rcm = rd.strand.astype(bool)
    comp = np.zeros(256, dtype=np.uint8)
    comp[list(b"ACGT")] = list(b"TGCA")
    fwd[rcm] = comp[reads[rcm][:, ::-1]]
    mism = (fwd != ref).reshape(n, 5, 20).any(axis=2)
    p_clean = 1.0 - mism.mean()
    v, tol = gold["p_seed_clean_2pct_s20"]
    assert abs(p_clean - v) < tol, p_clean
    p_all = mism.all(axis=1).mean()
    v, tol = gold["p_all5_dirty_2pct_s20"]
    assert abs(p_all - v) < tol, p_all


def test_chance_hits_scale_as_genome_over_4_to_the_s():
    # The paper's example: G ~ 4^16, s = 10 -> 4^6 chance hits, s = 20 -> 4^-4.
    # Same ratio here at a size a test can scan: G = 4^11 and s = 10 -> 4.
    gold = _golden()
    v10, t10 = gold["chance_hits_s10_g4pow16"]
    v20, t20 = gold["chance_hits_s20_g4pow16"]
    assert abs(4.0 ** 16 / 4.0 ** 10 - v10) < t10 and abs(4.0 ** 16 / 4.0 ** 20 - v20) < t20
    G = 4 ** 11
    g, _ = synth.genome(G, 0.0, seed_genome=99)
    idx = oracle.Index(g, 10)
    rng = np.random.default_rng(1)
    q = np.frombuffer(b"ACGT", dtype=np.uint8)[rng.integers(0, 4, (400, 10))]
    hits = [len(idx.occurrences(row.tobytes())) for row in q]
    expect = (G - 9) / 4.0 ** 10
    assert abs(np.mean(hits) - expect) < 0.5


def test_repeat_families_cover_target_fraction():
    G = 5_000_000
    g, cov = synth.genome(G, 0.05)
    assert 0.05 * G <= cov < 0.05 * G + 6000 * 1
    # repeats create 20-mers that occur many times; a uniform genome has almost none
    idx = oracle.Index(g[:1_000_000], 20)
    assert idx.entries == 1_000_000 - 19


def test_read_length_mixes():
    l1 = synth.read_lengths(200_000, 1, lo=100, hi=1000)
    assert l1.min() >= 100 and l1.max() <= 1000
    assert abs(l1.mean() - 900 / np.log(10)) < 5          # log-uniform mean (b - a)/ln(b/a)
    l2 = synth.read_lengths(200_000, 2, m_fixed=100, lo=1000, hi=10000, frac_fixed=0.8)
    assert abs((l2 == 100).mean() - 0.8) < 0.01
    assert abs(l2.mean() - (0.8 * 100 + 0.2 * 9000 / np.log(10))) < 15
