"""Pins for the oracle's Algorithm 1 ("SNAP alignment algorithm").

Each branch of Algorithm 1 gets a hand-built genome (uniform random background with
planted copies) and a read whose outcome is worked by hand from the pseudocode; the
derivation is in each test's comment.  Distances the derivation relies on are checked
first with the textbook table (itself pinned in test_oracle_ed.py).  Then the
invariants that hold on any input:

* error-free reads from unique sequence come back as a single hit at their origin
  with distance 0, on both strands;
* the reported distance equals the full-table distance at the reported location;
* the speculate-then-replay mode (every candidate scored once at d_max + c - 1, the
  decisions replayed with ED(L) = d0 if d0 <= L else over) equals the literal mode.
"""
import numpy as np
import pytest

import oracle
import synth

NF, SINGLE, MULTI = oracle.NOT_FOUND, oracle.SINGLE_HIT, oracle.MULTIPLE_HITS
S = 20


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    return bytearray(np.frombuffer(b"ACGT", dtype=np.uint8)[rng.integers(0, 4, n)].tobytes())


def _rc(a: bytes) -> bytes:
    return bytes(a)[::-1].translate(bytes.maketrans(b"ACGT", b"TGCA"))


def _sub(a: bytes, i: int) -> bytes:
    a = bytearray(a)
    a[i] = {ord("A"): ord("C"), ord("C"): ord("G"), ord("G"): ord("T"), ord("T"): ord("A")}[a[i]]
    return bytes(a)


def _align(genome: bytes, reads, **kw):
    idx = oracle.Index(np.frombuffer(bytes(genome), dtype=np.uint8), S)
    bases = np.frombuffer(b"".join(reads), dtype=np.uint8)
    offs = np.zeros(len(reads) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([len(r) for r in reads])
    params = dict(max_dist=8, max_hits=300, conf_diff=2, num_seeds=0)
    params.update(kw)
    res, st = idx.align(bases, offs, **params)
    res1, _ = idx.align(bases, offs, mode=1, **params)
    assert np.array_equal(res, res1), "replay mode disagrees with literal mode"
    return res, st


def _tup(r):
    return (int(r["location"]), int(r["strand"]), int(r["edit_distance"]), int(r["cls"]))


def test_error_free_unique_reads_single_at_origin_both_strands():
    g = bytes(_rand(20_000, 1))
    reads = [g[1000:1100], _rc(g[5000:5100]), g[19_900:20_000], _rc(g[0:100])]
    res, _ = _align(g, reads)
    assert [_tup(r) for r in res] == [(1000, 0, 0, SINGLE), (5000, 1, 0, SINGLE),
                                      (19_900, 0, 0, SINGLE), (0, 1, 0, SINGLE)]


def test_early_multiple_return():
    # Region A at 2000 copied exactly to 9000.  Seed 1 votes once for each; the
    # smaller key (2000, strand 0) is scored first with L = d_max+c-1: d = 0,
    # t = 1, no exit.  Seed 2 makes both 2 votes; 9000 is scored with
    # L = d_best+c-1 = 1: d = 0 in another bucket, so d_second = 0.  Now
    # d_best < c and d_second < d_best + c: return "multiple hits" at the
    # earliest-scored best, 2000.
    g = _rand(20_000, 2)
    g[9000:9100] = g[2000:2100]
    g = bytes(g)
    res, st = _align(g, [g[2000:2100]])
    assert _tup(res[0]) == (2000, 0, 0, MULTI)
    assert st.ed_calls == 2


def test_baeza_yates_stop_skips_later_candidates():
    # B at 12000 = A (at 3000) with substitutions at read offsets 10 and 30, so
    # seeds 1 and 2 hit only A, seeds 3-5 hit both.  Seed 1: A scored, d = 0,
    # t = 1.  Seed 2: nothing unscored, t = 2 >= d_best + c = 2: score what is
    # left (nothing) and stop.  B is never scored.
    g = _rand(20_000, 3)
    a = bytes(g[3000:3100])
    g[12000:12100] = _sub(_sub(a, 10), 30)
    g = bytes(g)
    assert oracle.ed_dp(a, g[12000:12200]) == 2
    res, st = _align(g, [a])
    assert _tup(res[0]) == (3000, 0, 0, SINGLE)
    assert st.ed_calls == 1


def test_drain_scores_every_remaining_candidate():
    # Seed 2 (offset 20) of the read also occurs at 8000 and 14000 inside random
    # sequence.  Seed 1: A (5000) scored, d = 0, t = 1.  Seed 2: C1 = 8000-20 and
    # C2 = 14000-20 have one vote each; the pick takes C1 (smaller key) with
    # L = 1 (over).  t = 2 >= 2: the drain scores C2 (over).  Three calls; the
    # result stays a single hit at A.  Without the drain C2 would not be scored.
    g = _rand(20_000, 4)
    a = bytes(g[5000:5100])
    g[8000:8020] = a[20:40]
    g[14000:14020] = a[20:40]
    g = bytes(g)
    res, st = _align(g, [a])
    assert _tup(res[0]) == (5000, 0, 0, SINGLE)
    assert st.ed_calls == 3 and st.ed_over == 2


def test_all_seeds_popular_is_multiple_and_hmax_boundary():
    # Every seed of the read occurs twice.  h_max = 1: all five seeds are
    # skipped, and "all seeds had > h_max entries" gives multiple hits with no
    # location.  h_max = 2 (count exactly h_max): the seeds are used and the
    # early-multiple path of test_early_multiple_return applies.
    g = _rand(20_000, 5)
    g[11000:11100] = g[1000:1100]
    g = bytes(g)
    res, st = _align(g, [g[1000:1100]], max_hits=1)
    assert _tup(res[0]) == (-1, 0, -1, MULTI)
    assert st.ed_calls == 0 and st.seeds_popular == 5
    res, _ = _align(g, [g[1000:1100]], max_hits=2)
    assert _tup(res[0]) == (1000, 0, 0, MULTI)


def test_not_found_and_short_reads():
    g = bytes(_rand(20_000, 6))
    foreign = bytes(_rand(100, 606))
    res, st = _align(g, [foreign, g[100:115]])
    assert _tup(res[0]) == (-1, 0, -1, NF)
    assert _tup(res[1]) == (-1, 0, -1, NF)   # shorter than a seed
    assert st.ed_calls == 0


def test_best_between_dmax_and_limit_is_not_reported():
    # d_max = 2, c = 2, so the first limit is d_max + c - 1 = 3.  Substitutions
    # at read offsets 25, 45, 65 spoil seeds 2-4; seeds 1 and 5 are exact.  Seed
    # 1: A scored with L = 3, d = 3 (a hit, but d_best > d_max).  Seeds 2-4 have
    # no hits but count toward t (2, 3, 4).  Seed 5: t = 5 >= d_best + c = 5:
    # stop.  Final: d_best > d_max and not all seeds popular: not found.  With
    # only two substitutions the same read is a single hit at distance 2.
    g = bytes(_rand(20_000, 7))
    a = g[7000:7100]
    r3 = _sub(_sub(_sub(a, 25), 45), 65)
    r2 = _sub(_sub(a, 25), 45)
    assert oracle.ed_dp(r3, g[7000:7200]) == 3 and oracle.ed_dp(r2, g[7000:7200]) == 2
    res, _ = _align(g, [r3, r2], max_dist=2)
    assert _tup(res[0]) == (-1, 0, -1, NF)
    assert _tup(res[1]) == (7000, 0, 2, SINGLE)


@pytest.mark.parametrize("p,expect_cls", [(32 * 100 + 5, SINGLE), (32 * 100 + 31, MULTI)])
def test_bucket_merge_of_indel_shifted_candidates(p, expect_cls):
    # Read = G[p..p+40) + G[p+41..p+101): one base deleted at read offset 40.
    # Seeds 1-2 vote for p, seeds 3-5 for p+1.  Seed 1: p scored, d = 1, t = 1.
    # Seed 3: p+1 scored with L = d_best + c - 1 = 2, d = 2.  If p and p+1 share
    # a 32-base bucket, p+1 does not count as a second-best: t reaches 3 >=
    # d_best + c and the read is a single hit at p.  If p = 31 (mod 32) they sit
    # in different buckets: d_second = 2 < d_best + c with d_best < c, so the
    # read returns multiple hits at p.
    g = bytes(_rand(40_000, 8))
    read = g[p:p + 40] + g[p + 41:p + 101]
    assert oracle.ed_dp(read, g[p:p + 200]) == 1
    assert oracle.ed_dp(read, g[p + 1:p + 200]) == 2
    res, st = _align(g, [read])
    assert _tup(res[0]) == (p, 0, 1, expect_cls)
    assert st.ed_calls == 2


def test_distance_tie_keeps_earliest_scored():
    # B (9000) = R with a substitution at offset 90, A (2000) = R with one at
    # offset 10.  Seed 1 hits only B: B scored first, d = 1.  Seed 2: A (1 vote)
    # is the unscored pick, L = 2, d = 1 in another bucket: d_best = 1 is kept
    # by B (scored first) although A has the smaller key; d_second = 1 < 3 and
    # d_best < c: multiple hits at B.
    g = _rand(20_000, 9)
    r = bytes(_rand(100, 909))
    g[2000:2100] = _sub(r, 10)
    g[9000:9100] = _sub(r, 90)
    g = bytes(g)
    res, _ = _align(g, [r])
    assert _tup(res[0]) == (9000, 0, 1, MULTI)


def test_palindromic_seed_votes_on_both_strands():
    # Seed 1 of the read is its own reverse complement, so it votes for
    # (strand 0, p) and (strand 1, p - 80) (l - (m - o - s) with o = 0).  The
    # strand-1 key 2(p-80)+1 is smaller, so it is scored first (over).  Seed 2
    # makes (p, 0) the unscored favourite: d = 0.  Single hit at p, two calls.
    g = _rand(20_000, 10)
    p = 6000
    pal = b"ACGTTGCAAG" + _rc(b"ACGTTGCAAG")
    assert pal == _rc(pal)
    g[p:p + 20] = pal
    g = bytes(g)
    res, st = _align(g, [g[p:p + 100]])
    assert _tup(res[0]) == (p, 0, 0, SINGLE)
    assert st.ed_calls == 2


def test_invariants_on_synthetic_workload():
    w = synth.CONFIGS["C1"].scaled(G=1_000_000, n_reads=4000, name="C1-4k")
    g, _ = w.make_genome()
    rd = w.make_reads(g)
    idx = oracle.Index(g, w.seed_len)
    res, st = idx.align(rd.bases, rd.offsets, **w.params())
    res1, _ = idx.align(rd.bases, rd.offsets, mode=1, **w.params())
    assert np.array_equal(res, res1)
    # reported distance == full table at the reported location
    xs, ts = [], []
    gb = g.tobytes()
    for i in np.nonzero(res["location"] >= 0)[0][:1500]:
        p = int(res["location"][i])
        r = rd.bases[rd.offsets[i]:rd.offsets[i + 1]].tobytes()
        if res["strand"][i]:
            r = _rc(r)
        xs.append(r)
        ts.append(gb[p:p + 2 * len(r)])
    _, dp = oracle.ed_pairs(xs, ts, [0] * len(xs))
    loc = np.nonzero(res["location"] >= 0)[0][:1500]
    assert np.array_equal(dp, res["edit_distance"][loc])
    # error-free reads from a uniform genome: single at origin, distance 0
    clean = synth.reads(g, np.full(500, 100, dtype=np.uint32), 0.0, 0.0, seed=77)
    cres, _ = idx.align(clean.bases, clean.offsets, **w.params())
    assert (cres["cls"] == SINGLE).all()
    assert np.array_equal(cres["location"], clean.origin)
    assert np.array_equal(cres["strand"], clean.strand)
    assert (cres["edit_distance"] == 0).all()
    # accuracy vs simulated truth (soft: SNAP is a heuristic)
    single = res["cls"] == SINGLE
    near = np.abs(res["location"] - rd.origin) <= 30
    assert single.mean() > 0.95 and (near & single).sum() / single.sum() > 0.99


@pytest.mark.parametrize("cfg,G,n", [("C2", 3_000_000, 3000), ("C3", 4_000_000, 1500)])
def test_replay_mode_and_filtered_index_agree(cfg, G, n):
    w = synth.CONFIGS[cfg].scaled(G=G, n_reads=n)
    g, _ = w.make_genome()
    rd = w.make_reads(g)
    dpr = w.max_dist_per_read(rd.lengths())
    full = oracle.Index(g, w.seed_len)
    r0, st = full.align(rd.bases, rd.offsets, max_dist_per_read=dpr, **w.params())
    r1, _ = full.align(rd.bases, rd.offsets, max_dist_per_read=dpr, mode=1, **w.params())
    assert np.array_equal(r0, r1)
    keys = oracle.read_seed_kmers(rd.bases, rd.offsets, w.seed_len, w.num_seeds)
    filt = oracle.Index(g, w.seed_len, kmer_filter=keys)
    r2, _ = filt.align(rd.bases, rd.offsets, max_dist_per_read=dpr, threads=4, **w.params())
    assert np.array_equal(r0, r2)
    assert st.n_single > 0.6 * n  # long indels (up to 20 bases) push some reads past d_max


def _align_first(genome: bytes, reads, first_seeds, **kw):
    idx = oracle.Index(np.frombuffer(bytes(genome), dtype=np.uint8), S)
    bases = np.frombuffer(b"".join(reads), dtype=np.uint8)
    offs = np.zeros(len(reads) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([len(r) for r in reads])
    params = dict(max_dist=8, max_hits=300, conf_diff=2, num_seeds=0, first_seeds=first_seeds)
    params.update(kw)
    res, st = idx.align(bases, offs, **params)
    res1, _ = idx.align(bases, offs, mode=1, **params)
    assert np.array_equal(res, res1), "replay mode disagrees with literal mode"
    return res, st


def test_seeds_first_variant_changes_the_outcome():
    # A 50 bp read has two seeds, at 0 and 20.  B (9000) is the read with one
    # substitution at base 45 (outside both seeds): d = 1, voted by both seeds.
    # A (2000) is the read with substitutions at 25 and 35: d = 2, voted by seed 0
    # only.
    # Algorithm 1 (first_seeds 0 or 1): after seed 0, A and B have one vote each and
    # the smaller key A is scored at L = d_max+c-1: d_best = 2.  After seed 1, B (two
    # votes) is scored at L = d_best+c-1 = 3: d = 1, so d_best = 1 and d_second = 2
    # (A, another bucket): d_best < c and d_second < d_best+c, return "multiple" at
    # B after two distance calls.
    # Seeds-first with k = 2 (or any k >= 2, the read having only two non-popular
    # seeds): both seeds vote first, B leads 2 to 1 and is scored: d_best = 1, no
    # second; no exit passes (t = 2 < d_best+c = 3) and the seeds run out, so the
    # read is a single hit at B after one call; A is never scored.
    g = _rand(20_000, 17)
    read = bytes(_rand(50, 18))
    g[9000:9050] = _sub(read, 45)
    g[2000:2050] = _sub(_sub(read, 25), 35)
    g = bytes(g)
    assert oracle.ed_dp(read, g[9000:9100]) == 1 and oracle.ed_dp(read, g[2000:2100]) == 2
    for k in (0, 1):
        res, st = _align_first(g, [read], k)
        assert _tup(res[0]) == (9000, 0, 1, MULTI) and st.ed_calls == 2
    for k in (2, 5):
        res, st = _align_first(g, [read], k)
        assert _tup(res[0]) == (9000, 0, 1, SINGLE) and st.ed_calls == 1


def test_seeds_first_one_equals_algorithm_1_on_workloads():
    # first_seeds 0 and 1 are both Algorithm 1; larger values differ only in order
    # and never find a distance that is not the table's at the reported location
    w = synth.CONFIGS["C2"].scaled(G=1_000_000, n_reads=3000)
    g, _ = w.make_genome()
    rd = w.make_reads(g)
    idx = oracle.Index(g, w.seed_len)
    base, _ = idx.align(rd.bases, rd.offsets, **w.params())
    one, _ = idx.align(rd.bases, rd.offsets, first_seeds=1, **w.params())
    assert np.array_equal(base, one)
    three, st3 = idx.align(rd.bases, rd.offsets, first_seeds=3, **w.params())
    replay, _ = idx.align(rd.bases, rd.offsets, first_seeds=3, mode=1, **w.params())
    assert np.array_equal(three, replay)
    hit = np.nonzero(three["location"] >= 0)[0][:200]
    for i in hit:
        x = bytes(rd.bases[rd.offsets[i]:rd.offsets[i + 1]])
        if three["strand"][i]:
            x = _rc(x)
        p = int(three["location"][i])
        assert oracle.ed_dp(x, bytes(g[p:p + len(x) + 20])) == three["edit_distance"][i]


@pytest.mark.parametrize("stride", [2, 3, 5])
def test_strided_index_error_free_reads_at_every_phase(stride):
    # With a stride-k index each seed is looked up at k consecutive offsets, so an
    # error-free read from unique sequence meets the index whatever its origin modulo
    # k: single hit at the origin with distance 0, on both strands.
    g = bytes(_rand(30_000, 21))
    idx = oracle.Index(np.frombuffer(g, dtype=np.uint8), S, stride=stride)
    reads, expect = [], []
    for q in range(stride):
        p = 1000 + 997 * q + q  # every residue of p modulo the stride
        reads += [g[p:p + 100], _rc(g[p + 5000:p + 5100])]
        expect += [(p, 0, 0, SINGLE), (p + 5000, 1, 0, SINGLE)]
    bases = np.frombuffer(b"".join(reads), dtype=np.uint8)
    offs = np.zeros(len(reads) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([len(r) for r in reads])
    res, st = idx.align(bases, offs, max_dist=8, max_hits=300, conf_diff=2)
    assert [_tup(r) for r in res] == expect
    # seeds at 0, 20, 40, 60 get k probes; the one at 80 has room for one (80 + 20 = m)
    assert st.seeds_looked_up == len(reads) * (4 * stride + 1)
    res1, _ = idx.align(bases, offs, max_dist=8, max_hits=300, conf_diff=2, mode=1)
    assert np.array_equal(res, res1)


def test_strided_index_workloads_stride_one_and_replay():
    # stride 1 is the plain index; for larger strides the replay mode equals the
    # literal one and every reported distance is the table's at the reported place
    w = synth.CONFIGS["C2"].scaled(G=1_000_000, n_reads=2000)
    g, _ = w.make_genome()
    rd = w.make_reads(g)
    base, _ = oracle.Index(g, w.seed_len).align(rd.bases, rd.offsets, **w.params())
    one, _ = oracle.Index(g, w.seed_len, stride=1).align(rd.bases, rd.offsets, **w.params())
    assert np.array_equal(base, one)
    for stride in (2, 4):
        idx = oracle.Index(g, w.seed_len, stride=stride)
        lit, st = idx.align(rd.bases, rd.offsets, **w.params())
        rep, _ = idx.align(rd.bases, rd.offsets, mode=1, **w.params())
        assert np.array_equal(lit, rep)
        assert (lit["cls"] == SINGLE).mean() > 0.85
        for i in np.nonzero(lit["location"] >= 0)[0][:150]:
            x = bytes(rd.bases[rd.offsets[i]:rd.offsets[i + 1]])
            if lit["strand"][i]:
                x = _rc(x)
            p = int(lit["location"][i])
            assert oracle.ed_dp(x, bytes(g[p:p + len(x) + 20])) == lit["edit_distance"][i]


def test_against_exhaustive_search_on_a_tiny_genome():
    # "Exhaustive SNAP": the bounded distance of every read at every genome position on
    # both strands.  Exact check: a reported hit's distance is the exhaustive table's at
    # its (p, strand).  Soft check (SNAP is a heuristic and only scores what its seeds
    # vote for): at least 90% of the confident hits reach the exhaustive optimum.
    rng = np.random.default_rng(31)
    g = _rand(5000, 31)
    for src, dst in ((200, 3000), (1200, 4200)):  # near repeats at 2% divergence
        unit = bytearray(g[src:src + 300])
        for i in rng.choice(300, 6, replace=False):
            unit[i] = b"ACGT"[(b"ACGT".index(unit[i]) + 1) % 4]
        g[dst:dst + 300] = unit
    g = bytes(g)
    reads = []
    for k in range(60):
        p = int(rng.integers(0, 5000 - 80))
        r = bytearray(g[p:p + 60])
        for i in rng.choice(60, int(rng.integers(0, 3)), replace=False):
            r[i] = b"ACGT"[(b"ACGT".index(r[i]) + 1) % 4]
        reads.append(bytes(r) if k % 2 == 0 else _rc(bytes(r)))
    d_max, c = 8, 2
    res, _ = _align(g, reads, max_dist=d_max, conf_diff=c)
    L = d_max + c - 1
    agree = confident = 0
    for r, x in zip(res, reads):
        X = [x, _rc(x)]
        xs = [X[st] for st in (0, 1) for p in range(len(g))]
        ts = [g[p:p + len(x) + L] for st in (0, 1) for p in range(len(g))]
        lv, _ = oracle.ed_pairs(xs, ts, [L] * len(xs), with_dp=False)
        d = np.where(lv < 0, 10_000, lv).reshape(2, len(g))
        if r["location"] >= 0:
            assert d[int(r["strand"]), int(r["location"])] == r["edit_distance"]
        if r["cls"] == SINGLE:
            confident += 1
            agree += int(r["edit_distance"] == d.min())
    assert confident >= 40 and agree / confident >= 0.9
