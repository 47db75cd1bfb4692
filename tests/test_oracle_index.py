"""Pins for the oracle's seed index and seed order.

Index ("Hash Index" subsection): every overlapping s-mer of the genome is indexed
(window slid one base at a time).  Pinned against a brute-force scan of every genome
position written with numpy, including palindromic seeds and the last window.

Seed order (item 3 of the list after Algorithm 1): pinned against every offset of
three shapes worked by hand from the paper's wording (tests/golden/seed_order_*.txt:
m = 100 / s = 20, m = 64 / s = 16, m = 50 / s = 12) and against invariants that hold
for any (m, s): every offset in [0, m-s] used exactly once, the first floor(m/s)
offsets are the non-overlapping ones, and the passes spread out level by level: once
the shifts of the halving levels up to k (s/2, then s/4 and 3s/4, ...) are all used,
they are 2^k points that cut [0, s) into gaps of floor(s/2^k) or ceil(s/2^k) bases,
the most even spacing integers allow.
"""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_ints(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [int(x) for line in f if not line.startswith("#") for x in line.split()]


def _rand_genome(n, seed):
    rng = np.random.default_rng(seed)
    return np.frombuffer(b"ACGT", dtype=np.uint8)[rng.integers(0, 4, n)]


def _revcomp(a: bytes) -> bytes:
    return a[::-1].translate(bytes.maketrans(b"ACGT", b"TGCA"))


@pytest.mark.parametrize("m,s,name", [(100, 20, "seed_order_m100_s20.txt"),
                                      (64, 16, "seed_order_m64_s16.txt"),
                                      (50, 12, "seed_order_m50_s12.txt")])
def test_seed_order_matches_hand_worked_offsets(m, s, name):
    expect = _golden_ints(name)
    assert len(expect) == m - s + 1  # the golden files list every window
    offs, pass0 = oracle.seed_offsets(m, s, 10 ** 6)
    assert offs == expect
    k = m // s
    assert pass0 == [True] * k + [False] * (len(expect) - k)
    # any prefix is the first n seeds
    for n in (1, k, k + 1, 17, len(expect) - 1):
        assert oracle.seed_offsets(m, s, n)[0] == expect[:n]


def _pass_shifts(s):
    """Shift of every pass, in order: the first offset of each pass of a read long
    enough that every pass has one (a pass starts below s, later offsets do not)."""
    offs, _ = oracle.seed_offsets(4 * s, s, 10 ** 6)
    return [o for o in offs if o < s]


@pytest.mark.parametrize("s", [8, 12, 16, 17, 20, 24, 31, 32])
def test_seed_passes_spread_out_level_by_level(s):
    shifts = _pass_shifts(s)
    assert sorted(shifts) == list(range(s))  # every shift once
    assert shifts[0] == 0 and shifts[1] == s // 2
    k = 1
    while (1 << k) <= s:
        used = sorted(shifts[:1 << k]) + [s]
        gaps = {b - a for a, b in zip(used, used[1:])}
        assert gaps <= {s >> k, -(-s >> k)}, (k, used)
        k += 1


@pytest.mark.parametrize("m,s", [(100, 20), (125, 20), (37, 8), (1000, 20), (64, 32),
                                 (20, 20), (19, 20), (333, 17)])
def test_seed_order_invariants(m, s):
    offs, pass0 = oracle.seed_offsets(m, s, 10 ** 6)
    if m < s:
        assert offs == []
        return
    assert sorted(offs) == list(range(m - s + 1))  # every window once
    k = m // s
    assert offs[:k] == [i * s for i in range(k)]   # sequential non-overlapping first
    assert all(pass0[:k]) and not any(pass0[k:])
    # default n = floor(m/s): exactly the non-overlapping pass
    d_offs, _ = oracle.seed_offsets(m, s, m // s)
    assert d_offs == offs[:k]
    # the second pass is shifted by floor(s/2)
    if m - s >= s // 2 and s >= 2:
        assert offs[k] == s // 2


def _brute_positions(g: bytes, smer: bytes):
    s = len(smer)
    return [l for l in range(len(g) - s + 1) if g[l:l + s] == smer]


def test_index_matches_brute_force_scan():
    s = 12
    g = bytearray(_rand_genome(20_000, 5).tobytes())
    # plant repeats, a palindrome (ACGTTAACGT... is its own reverse complement) and
    # a window at the very end
    unit = bytes(g[100:140])
    for pos in (3000, 7000, 15000):
        g[pos:pos + 40] = unit
    pal = b"ACGTAC" + _revcomp(b"ACGTAC")
    assert pal == _revcomp(pal)
    for pos in (500, 9000):
        g[pos:pos + s] = pal
    g = bytes(g)
    idx = oracle.Index(np.frombuffer(g, dtype=np.uint8), s)
    assert idx.entries == len(g) - s + 1
    queries = [g[100:100 + s], g[110:110 + s], pal, g[len(g) - s:], g[0:s]]
    rng = np.random.default_rng(9)
    for _ in range(300):
        l = int(rng.integers(0, len(g) - s + 1))
        queries.append(g[l:l + s])
    for _ in range(100):  # mostly absent keys
        queries.append(bytes(_rand_genome(s, int(rng.integers(1 << 30))).tobytes()))
    for q in queries:
        assert idx.occurrences(q) == _brute_positions(g, q), q
    assert len(idx.occurrences(pal)) == 2
    assert len(idx.occurrences(g[100:100 + s])) == 4


def test_filtered_index_keeps_exactly_the_filter():
    s = 10
    g = _rand_genome(5000, 6)
    full = oracle.Index(g, s)
    # reads = a few windows; filter = their seed s-mers and reverse complements
    gb = g.tobytes()
    reads = [gb[100:150], gb[2000:2050], _revcomp(gb[3000:3050])]
    bases = np.frombuffer(b"".join(reads), dtype=np.uint8)
    offs = np.array([0, 50, 100, 150], dtype=np.uint64)
    keys = oracle.read_seed_kmers(bases, offs, s, 0)
    filt = oracle.Index(g, s, kmer_filter=keys)
    for r in reads:
        for o in range(0, 50 - s + 1, s):
            q = r[o:o + s]
            assert filt.occurrences(q) == full.occurrences(q)
            assert filt.occurrences(_revcomp(q)) == full.occurrences(_revcomp(q))
    assert filt.entries < full.entries


def test_index_rejects_bad_input():
    with pytest.raises(ValueError):
        oracle.Index(np.frombuffer(b"ACGTNACGTACGTACGTACGT", dtype=np.uint8), 8)
    with pytest.raises(ValueError):
        oracle.Index(np.frombuffer(b"ACGT", dtype=np.uint8), 8)


@pytest.mark.parametrize("stride", [2, 3, 4])
def test_strided_index_matches_brute_force_scan(stride):
    # stride-k index (Overlapping Seeds footnote): exactly the windows starting at a
    # multiple of k, every other window absent
    s = 12
    g = bytearray(_rand_genome(20_000, 6).tobytes())
    unit = bytes(g[100:140])
    for pos in (3001, 7002, 15003):
        g[pos:pos + 40] = unit
    g = bytes(g)
    idx = oracle.Index(np.frombuffer(g, dtype=np.uint8), s, stride=stride)
    assert idx.entries == (len(g) - s) // stride + 1
    rng = np.random.default_rng(10)
    queries = [g[100:100 + s], g[101:101 + s], g[len(g) - s:], g[0:s]]
    for _ in range(300):
        l = int(rng.integers(0, len(g) - s + 1))
        queries.append(g[l:l + s])
    for q in queries:
        assert idx.occurrences(q) == [p for p in _brute_positions(g, q) if p % stride == 0], q
