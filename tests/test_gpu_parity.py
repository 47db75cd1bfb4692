"""Parity of the CUDA path with the oracle (bit-exact in every result field).

Every call goes through the C-ABI.  Workloads are the seeded synthetic recipes of
synth.CONFIGS (scaled where the oracle must finish in seconds) plus the hand-built
Algorithm 1 branch cases of test_oracle_align.py and edge cases (empty batch, reads
shorter than a seed, seed lengths 8 and 32, ragged lengths, bad bases).
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

FIELDS = ("location", "edit_distance", "strand", "cls")


@pytest.fixture(scope="module")
def snap():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1111_5572_gb300 as m
    return m


def assert_same(got, ref, what=""):
    for f in FIELDS:
        if not np.array_equal(got[f], ref[f]):
            bad = np.nonzero(got[f] != ref[f])[0]
            i = int(bad[0])
            raise AssertionError(f"{what}: field {f} differs at {len(bad)} reads, first {i}: "
                                 f"gpu={got[i]} oracle={ref[i]}")


def _run_both(snap, g, rd, w, plain=False, dpr=None, **kw):
    params = w.params()
    params.update(kw)
    gi = snap.Index(g, w.seed_len)
    got = gi.align(rd.bases, rd.offsets, max_dist_per_read=dpr, plain=plain, **params)
    ref, st = oracle.Index(g, w.seed_len).align(rd.bases, rd.offsets, max_dist_per_read=dpr,
                                                threads=4, **params)
    return got, ref, st


@pytest.mark.parametrize("plain", [False, True])
def test_c1_tiny_full(snap, plain):
    w = synth.CONFIGS["C1"]
    g, _ = w.make_genome()
    rd = w.make_reads(g)
    got, ref, st = _run_both(snap, g, rd, w, plain=plain)
    assert_same(got, ref, f"C1 plain={plain}")
    assert st.n_single > 9000


@pytest.mark.parametrize("plain", [False, True])
@pytest.mark.parametrize("G,n", [(3_000_000, 20_000)])
def test_c2_repeat_rich_scaled(snap, G, n, plain):
    w = synth.CONFIGS["C2"].scaled(G=G, n_reads=n)
    g, _ = w.make_genome()
    rd = w.make_reads(g)
    got, ref, st = _run_both(snap, g, rd, w, plain=plain)
    assert_same(got, ref, f"C2 scaled plain={plain}")
    assert st.n_multiple > 0  # the repeat families exercise the multiple-hit paths


def test_c5_repeat_dense_scaled(snap):
    # C5 recipe (50% of the genome in repeat families) on 10 Mbp: reads with dozens of
    # candidates, scored mostly in the drain, where the warp kernel ranks them and
    # scores 32 at a time (the limit can grow there: a new best in the old best's
    # 32-base bucket can lift d_second clear of it)
    w = synth.CONFIGS["C5"].scaled(G=10_000_000, n_reads=60_000)
    g, _ = w.make_genome()
    rd = w.make_reads(g)
    got, ref, st = _run_both(snap, g, rd, w)
    assert_same(got, ref, "C5 scaled")
    assert st.n_multiple > 1000


def test_exact_duplicate_collapsing(snap):
    """Exact-duplicate collapsing (Ongoing Work, Approach): on a genome whose repeat
    copies are exact, the parallel drain finds candidates with identical windows and
    computes each distinct window's distance once; every result equals the run without
    collapsing and the oracle's."""
    G = 5_000_000
    g, _ = synth.genome(G, 0.3, divergence=0.0)
    w = synth.CONFIGS["C5"].scaled(G=G, n_reads=30_000)
    rd = synth.reads(g, np.full(30_000, 100, dtype=np.uint32), w.sub_rate, w.indel_rate,
                     w.indel_len, seed=31)
    gi = snap.Index(g, w.seed_len)
    off = gi.align(rd.bases, rd.offsets, **w.params())
    assert gi.last_call_stats()["ed_collapsed"] == 0
    on = gi.align(rd.bases, rd.offsets, collapse_duplicates=1, **w.params())
    st = gi.last_call_stats()
    assert st["ed_collapsed"] > 1000, st["ed_collapsed"]
    assert_same(on, off, "collapsing on vs off")
    ref, _ = oracle.Index(g, w.seed_len).align(rd.bases, rd.offsets, threads=16, **w.params())
    assert_same(on, ref, "collapsing vs oracle")
    with pytest.raises(snap.SnapError):
        gi.align(rd.bases[:100], rd.offsets[:2], collapse_duplicates=2, **w.params())


@pytest.mark.parametrize("h_max", [30, 3000])
def test_hmax_sweep_points(snap, h_max):
    # the h_max sweep's end points on the repeat-dense recipe (seeds hitting 30-3000
    # places: popular seeds, long vote lists, many candidates per read)
    w = replace(synth.CONFIGS["C5"].scaled(G=10_000_000, n_reads=20_000), max_hits=h_max)
    g, _ = w.make_genome()
    rd = w.make_reads(g)
    got, ref, st = _run_both(snap, g, rd, w)
    assert_same(got, ref, f"C5 scaled h_max={h_max}")
    if h_max == 30:
        assert st.seeds_popular > 0


@pytest.mark.parametrize("plain", [False, True])
def test_c3_uneven_lengths_scaled(snap, plain):
    w = synth.CONFIGS["C3"].scaled(G=4_000_000, n_reads=4000)
    g, _ = w.make_genome()
    rd = w.make_reads(g)
    dpr = w.max_dist_per_read(rd.lengths())
    got, ref, _ = _run_both(snap, g, rd, w, dpr=dpr, plain=plain)
    assert_same(got, ref, f"C3 scaled plain={plain}")


@pytest.mark.parametrize("plain", [False, True])
def test_c3_uneven_lengths_40Mbp_50k(snap, plain):
    """The C3 recipe at 40 Mbp with 50,000 reads: enough reads per length class that
    the batch-size-driven launch choices (warp per read for every class, the tuned
    shape) are those of the full 400 Mbp / 2M-read batch."""
    w = synth.CONFIGS["C3"].scaled(G=40_000_000, n_reads=50_000)
    g, _ = w.make_genome()
    rd = w.make_reads(g)
    dpr = w.max_dist_per_read(rd.lengths())
    params = w.params()
    gi = snap.Index(g, w.seed_len)
    got = gi.align(rd.bases, rd.offsets, max_dist_per_read=dpr, plain=plain, **params)
    if not plain:
        assert gi.last_call_stats()["team_classes"] == 0
    ref, st = oracle.Index(g, w.seed_len).align(rd.bases, rd.offsets, max_dist_per_read=dpr,
                                                threads=16, **params)
    assert_same(got, ref, f"C3 40 Mbp plain={plain}")
    assert st.n_single > 30_000


@pytest.mark.parametrize("plain", [False, True])
def test_c4_long_reads_scaled(snap, plain):
    # lengths: 80% 100 bp, 20% log-uniform [1000, 10000]; d_max = max(8, ceil(0.08 m))
    # reaches 800, which takes the shared-memory diagonal path of the edit distance
    w = synth.CONFIGS["C4"].scaled(G=2_000_000, n_reads=300)
    g, _ = w.make_genome()
    rd = w.make_reads(g, n=300)
    dpr = w.max_dist_per_read(rd.lengths())
    assert dpr.max() > 127
    got, ref, _ = _run_both(snap, g, rd, w, dpr=dpr, plain=plain)
    assert_same(got, ref, f"C4 scaled plain={plain}")


@pytest.mark.parametrize("s", [8, 12, 31, 32])
def test_seed_length_range(snap, s):
    w = synth.CONFIGS["C1"].scaled(G=300_000, n_reads=2000)
    w = replace(w, seed_len=s, num_seeds=0, max_hits=50)
    g, _ = w.make_genome()
    rd = w.make_reads(g)
    got, ref, _ = _run_both(snap, g, rd, w)
    assert_same(got, ref, f"s={s}")


def test_ragged_and_degenerate_reads(snap):
    g, _ = synth.genome(500_000, 0.05)
    lens = np.array([0, 1, 19, 20, 21, 39, 40, 100, 101, 257, 1000, 5, 64, 65, 1023, 1024],
                    dtype=np.uint32)
    lens = np.concatenate([lens, np.random.default_rng(1).integers(0, 600, 500).astype(np.uint32)])
    rd = synth.reads(g, lens, 0.02, 0.005, (1, 8), seed=5)
    w = synth.CONFIGS["C1"]
    for kw in (dict(), dict(num_seeds=17), dict(num_seeds=2047), dict(max_hits=0),
               dict(max_hits=1), dict(max_dist=0, conf_diff=1), dict(conf_diff=5)):
        for plain in (False, True):
            got, ref, _ = _run_both(snap, g, rd, w, plain=plain, **kw)
            assert_same(got, ref, f"ragged {kw} plain={plain}")


def test_hand_built_branch_cases(snap):
    # the genomes of test_oracle_align.py, all reads in one batch
    rng = np.random.default_rng(2)
    g = bytearray(np.frombuffer(b"ACGT", dtype=np.uint8)[rng.integers(0, 4, 60_000)].tobytes())
    rc = lambda a: bytes(a)[::-1].translate(bytes.maketrans(b"ACGT", b"TGCA"))

    def sub(a, i):
        a = bytearray(a)
        a[i] = b"CGTA"[b"ACGT".index(a[i])]
        return bytes(a)

    g[9000:9100] = g[2000:2100]                       # exact repeat: early multiple
    a = bytes(g[3000:3100])
    g[12000:12100] = sub(sub(a, 10), 30)              # Baeza-Yates stop
    b = bytes(g[5000:5100])
    g[18000:18020] = b[20:40]
    g[24000:24020] = b[20:40]                         # drain
    g[31000:31100] = g[1000:1100]                     # popular with h_max = 1
    r = bytes(np.frombuffer(b"ACGT", dtype=np.uint8)[rng.integers(0, 4, 100)].tobytes())
    g[40000:40100] = sub(r, 10)
    g[47000:47100] = sub(r, 90)                       # distance tie
    pal = b"ACGTTGCAAG" + rc(b"ACGTTGCAAG")
    g[52000:52020] = pal                              # palindromic seed
    g = bytes(g)
    p1, p2 = 32 * 700 + 5, 32 * 800 + 31
    reads = [g[2000:2100], a, b, g[1000:1100], r, g[52000:52100],
             g[p1:p1 + 40] + g[p1 + 41:p1 + 101], g[p2:p2 + 40] + g[p2 + 41:p2 + 101],
             sub(sub(sub(g[7000:7100], 25), 45), 65), rc(g[100:200]), g[59_900:60_000],
             g[10:25], bytes(np.frombuffer(b"ACGT", dtype=np.uint8)[rng.integers(0, 4, 100)])]
    bases = np.frombuffer(b"".join(reads), dtype=np.uint8)
    offs = np.zeros(len(reads) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([len(x) for x in reads])
    gi = snap.Index(np.frombuffer(g, dtype=np.uint8), 20)
    oi = oracle.Index(np.frombuffer(g, dtype=np.uint8), 20)
    for kw in (dict(max_dist=8, max_hits=300, conf_diff=2), dict(max_dist=2, max_hits=1,
                                                                 conf_diff=2),
               dict(max_dist=8, max_hits=2, conf_diff=2)):
        for plain in (False, True):
            got = gi.align(bases, offs, plain=plain, **kw)
            ref, _ = oi.align(bases, offs, **kw)
            assert_same(got, ref, f"branch cases {kw}")


def test_seeds_first_variant(snap):
    # the hand-worked case of test_oracle_align.py (a 50 bp read: "multiple" under
    # Algorithm 1, "single" when both seeds vote first) in all three kernels of the
    # batched form (thread per read, warp per read after a give-up, team mode is for
    # long reads and tested below) and the plain form; then whole workloads
    g = bytearray(np.frombuffer(b"ACGT", dtype=np.uint8)[
        np.random.default_rng(17).integers(0, 4, 20_000)].tobytes())
    read = bytes(np.frombuffer(b"ACGT", dtype=np.uint8)[
        np.random.default_rng(18).integers(0, 4, 50)].tobytes())

    def sub(a, i):
        a = bytearray(a)
        a[i] = b"CGTA"[b"ACGT".index(a[i])]
        return bytes(a)

    g[9000:9050] = sub(read, 45)
    g[2000:2050] = sub(sub(read, 25), 35)
    gn = np.frombuffer(bytes(g), dtype=np.uint8)
    gi = snap.Index(gn, 20)
    bases = np.frombuffer(read, dtype=np.uint8)
    offs = np.array([0, 50], dtype=np.uint64)
    for k, cls in ((0, 2), (1, 2), (2, 1), (5, 1)):
        for plain in (False, True):
            got = gi.align(bases, offs, plain=plain, first_seeds=k)
            assert (int(got["location"][0]), int(got["cls"][0])) == (9000, cls), (k, plain)
    with pytest.raises(snap.SnapError):
        gi.align(bases, offs, first_seeds=-1)
    for name, G, n, dpr_rule in (("C2", 3_000_000, 20_000, False), ("C5", 10_000_000, 30_000, False),
                                 ("C4", 2_000_000, 300, True)):
        w = synth.CONFIGS[name].scaled(G=G, n_reads=n)
        g2, _ = w.make_genome()
        rd = w.make_reads(g2, n=n)
        dpr = w.max_dist_per_read(rd.lengths()) if dpr_rule else None
        for k in (3, 5):
            for plain in (False, True):
                got, ref, _ = _run_both(snap, g2, rd, w, plain=plain, dpr=dpr, first_seeds=k)
                assert_same(got, ref, f"{name} first_seeds={k} plain={plain}")


@pytest.mark.parametrize("stride", [2, 3])
def test_stride_k_index(snap, stride):
    # stride-k index (only windows at multiples of k; each seed probed at k offsets):
    # both forms against the oracle with the same stride, on short reads (C2 recipe),
    # uneven lengths with per-read limits (C3 recipe: probes near the read end are cut)
    # and the repeat-dense C5 recipe, plus the error-free phase case of the oracle pins
    for name, G, n in (("C2", 3_000_000, 20_000), ("C3", 4_000_000, 3000),
                       ("C5", 10_000_000, 20_000)):
        w = synth.CONFIGS[name].scaled(G=G, n_reads=n)
        g, _ = w.make_genome()
        rd = w.make_reads(g)
        dpr = w.max_dist_per_read(rd.lengths())
        gi = snap.Index(g, w.seed_len, stride=stride)
        info = gi.info()
        assert info["stride"] == stride
        ref, st = oracle.Index(g, w.seed_len, stride=stride).align(
            rd.bases, rd.offsets, max_dist_per_read=dpr, threads=4, **w.params())
        for plain in (False, True):
            got = gi.align(rd.bases, rd.offsets, max_dist_per_read=dpr, plain=plain,
                           **w.params())
            assert_same(got, ref, f"{name} stride={stride} plain={plain}")
        assert gi.last_call_stats()["seeds"] == st.seeds_looked_up
    g = np.frombuffer(b"ACGT", dtype=np.uint8)[np.random.default_rng(3).integers(0, 4, 100)]
    for bad in (0, 17):
        with pytest.raises(snap.SnapError):
            snap.Index(np.tile(g, 100), 20, stride=bad)


def test_autotune_and_graph_replay_keep_results(snap):
    # launch shapes and graph replay must never change a result: compare against the
    # untuned, ungraphed run on several batch sizes, through the graph update path
    import torch
    w = synth.CONFIGS["C2"].scaled(G=3_000_000, n_reads=30_000)
    g, _ = w.make_genome()
    rd = w.make_reads(g)
    gi = snap.Index(g, w.seed_len)
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream()
    d_b = torch.from_numpy(rd.bases).to(dev)
    d_o = torch.from_numpy(rd.offsets.view(np.int64)).to(dev)

    def run(n):
        out = torch.zeros((n, 16), dtype=torch.uint8, device=dev)
        gi.align_device(d_b, d_o[:n + 1], out, stream=stream, **w.params())
        stream.synchronize()
        return out.cpu().numpy().view(snap.RESULT_DTYPE).reshape(-1), gi.last_call_stats()

    gi.configure(autotune=False, cuda_graphs=False)
    refs = {n: run(n)[0] for n in (30_000, 20_000, 9_000)}
    gi.configure(autotune=True, cuda_graphs=True)
    shapes = set()
    for n in (30_000, 30_000, 20_000, 9_000, 30_000):
        got, st = run(n)
        assert_same(got, refs[n], f"tuned/graph n={n}")
        assert st["graph_replay"] == 1
        shapes.add((st["light_threads"], st["warps_per_block"], st["table_slots"]))
    assert all(t in (64, 128, 256) for t, _, _ in shapes)
    ref_oracle, _ = oracle.Index(g, w.seed_len).align(rd.bases, rd.offsets, threads=4,
                                                      **w.params())
    assert_same(refs[30_000], ref_oracle, "untuned vs oracle")


def test_empty_batch_and_bad_input(snap):
    g, _ = synth.genome(100_000, 0.0)
    gi = snap.Index(g, 20)
    out = gi.align(np.zeros(0, dtype=np.uint8), np.zeros(1, dtype=np.uint64))
    assert out.shape == (0,)
    bad = np.frombuffer(b"ACGTACGTNNACGTACGTACGTACGT", dtype=np.uint8)
    with pytest.raises(snap.SnapError) as e:
        gi.align(bad, np.array([0, bad.shape[0]], dtype=np.uint64))
    assert e.value.code == snap.SNAP_E_INVAL
    lower = np.frombuffer(b"acgtacgtacgtacgtacgtacgt", dtype=np.uint8)
    with pytest.raises(snap.SnapError):
        gi.align(lower, np.array([0, lower.shape[0]], dtype=np.uint64))
    with pytest.raises(snap.SnapError):
        gi.align(g[:100], np.array([0, 100], dtype=np.uint64), max_hits=70000)
    with pytest.raises(snap.SnapError):
        gi.align(g[:100], np.array([0, 100], dtype=np.uint64), conf_diff=0)
    with pytest.raises(snap.SnapError):
        gi.align(g[:100], np.array([50, 10], dtype=np.uint64))
    # the index still works after the failed calls
    got = gi.align(g[:100], np.array([0, 100], dtype=np.uint64))
    assert int(got["cls"][0]) == snap.SINGLE_HIT and int(got["location"][0]) == 0
    with pytest.raises(snap.SnapError):
        snap.Index(np.frombuffer(b"ACGTN" * 10, dtype=np.uint8), 20)


def test_index_info(snap):
    w = synth.CONFIGS["C2"].scaled(G=2_000_000, n_reads=10)
    g, _ = w.make_genome()
    gi = snap.Index(g, 20)
    inf = gi.info()
    npos = 2_000_000 - 19
    assert inf["genome_len"] == 2_000_000 and inf["seed_len"] == 20
    assert inf["table_slots"] >= npos * 3 // 2
    # every window's canonical s-mer is in the table; repeats share slots
    assert 0.9 * npos < inf["distinct_seeds"] <= npos
    # out-of-line entries = windows whose key occurs 2..65534 times
    oi = oracle.Index(g, 20)
    assert inf["list_entries"] <= npos


def test_device_entry_point_on_torch_stream(snap):
    import torch
    w = synth.CONFIGS["C1"].scaled(G=500_000, n_reads=5000)
    g, _ = w.make_genome()
    rd = w.make_reads(g)
    gi = snap.Index(g, 20)
    dev = torch.device("cuda:0")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        d_b = torch.from_numpy(rd.bases).to(dev, non_blocking=False)
        d_o = torch.from_numpy(rd.offsets.view(np.int64)).to(dev)
        d_out = torch.zeros((rd.n, 16), dtype=torch.uint8, device=dev)
    s.synchronize()
    gi.align_device(d_b, d_o, d_out, stream=s, **w.params())
    got = d_out.cpu().numpy().view(snap.RESULT_DTYPE).reshape(-1)
    ref, _ = oracle.Index(g, 20).align(rd.bases, rd.offsets, **w.params())
    assert_same(got, ref, "device entry point")
    # unaligned read start: offsets into the middle of the buffer
    sub = np.arange(1, rd.n)
    offs2 = rd.offsets[1:].copy()
    got2 = gi.align(rd.bases, offs2, **w.params())
    assert_same(got2, ref[1:], "offset base not 16-aligned")


def test_c2_full_size_sampled(snap):
    """The benchmark workload (100 Mbp, 5% repeats, 1M x 100 bp) in the launch the bench
    times; the oracle checks a sample of 20,000 reads with an index restricted to the
    seeds those reads look up."""
    w = synth.CONFIGS["C2"]
    g, _ = w.make_genome()
    rd = w.make_reads(g)
    gi = snap.Index(g, w.seed_len)
    got = gi.align(rd.bases, rd.offsets, **w.params())
    sample = np.sort(np.random.default_rng(42).choice(rd.n, 20_000, replace=False))
    sub = rd.subset(sample)
    keys = oracle.read_seed_kmers(sub.bases, sub.offsets, w.seed_len, w.num_seeds)
    oi = oracle.Index(g, w.seed_len, kmer_filter=keys)
    ref, st = oi.align(sub.bases, sub.offsets, threads=8, **w.params())
    assert_same(got[sample], ref, "C2 full-size sample")
    # properties that hold for every read: classes valid, located hits within d_max
    assert set(np.unique(got["cls"]).tolist()) <= {0, 1, 2}
    loc = got["location"] >= 0
    assert (got["edit_distance"][loc] <= w.max_dist).all()
    assert (got["location"][loc] < w.G).all()
    assert ((got["location"] == -1) == (got["edit_distance"] == -1)).all()


def test_team_mode_equals_warp_mode(snap):
    # Reads of 2.5-4 kb fall in one length class with limits up to 320.  The same
    # batch aligned with one warp per read (team=0), in team mode (team=1: a block
    # per read, all its warps on each edit distance), in wave mode (team=2: a block
    # per read, each warp on its own candidate of the next picks) and with the
    # per-batch choice (team=-1, team mode here) gives identical results, and the
    # oracle agrees on a sample.
    w = synth.CONFIGS["C4"].scaled(G=3_000_000, n_reads=0)
    g, _ = w.make_genome()
    gi = snap.Index(g, w.seed_len)
    n = 600
    lens = np.random.default_rng(7).integers(2500, 4001, n).astype(np.uint32)
    rd = synth.reads(g, lens, w.sub_rate, w.indel_rate, w.indel_len, seed=17)
    dpr = w.max_dist_per_read(rd.lengths())
    runs = {}
    for team in (0, 1, 2, -1):
        gi.configure(team=team)
        runs[team] = gi.align(rd.bases, rd.offsets, max_dist_per_read=dpr, **w.params())
        st = gi.last_call_stats()
        assert st["team_classes"] == (0 if team == 0 else 1), team
        assert st["wave_classes"] == (1 if team == 2 else 0), team
        assert st["ed_filtered"] > 0
        if team == 2:
            assert st["wave_warps"] in (2, 4, 8), st["wave_warps"]
    gi.configure(team=-1)
    assert_same(runs[1], runs[0], "team vs warp mode")
    assert_same(runs[2], runs[0], "wave vs warp mode")
    assert_same(runs[-1], runs[0], "chosen vs warp mode")
    with pytest.raises(snap.SnapError):
        gi.configure(team=3)
    j = 40
    ref, _ = oracle.Index(g, w.seed_len).align(rd.bases[:int(rd.offsets[j])], rd.offsets[:j + 1],
                                               max_dist_per_read=dpr[:j], threads=4, **w.params())
    assert_same(runs[1][:j], ref, "team mode vs oracle")
    assert_same(runs[2][:j], ref, "wave mode vs oracle")


@pytest.mark.parametrize("case", ["low_error", "exact_copies"])
def test_wave_mode_exits(snap, case):
    # Wave mode takes Algorithm 1's steps ahead of their scores, so its exits are
    # the cases to check: reads of 1-2 kb with 0.3% errors meet the Baeza-Yates test
    # (t >= d_best + c) a few seeds in, usually inside a wave, whose later steps are
    # then undone before the drain; on a genome of exact repeat copies, error-free
    # reads in copies end early (d_best < c and a second hit within c).  Wave mode
    # = warp mode = team mode = oracle, read for read.
    w = synth.CONFIGS["C4"].scaled(G=3_000_000, n_reads=0)
    if case == "low_error":
        g, _ = w.make_genome()
        sub, indel = 0.003, 0.0005
    else:
        g, _ = synth.genome(3_000_000, 0.5, divergence=0.0)
        sub, indel = 0.0, 0.0
    gi = snap.Index(g, w.seed_len)
    n = 400
    lens = np.random.default_rng(11).integers(1000, 2001, n).astype(np.uint32)
    rd = synth.reads(g, lens, sub, indel, w.indel_len, seed=23)
    dpr = w.max_dist_per_read(rd.lengths())
    assert dpr.min() > 31  # every read in a block-per-read class
    runs = {}
    try:
        for team in (0, 1, 2):
            gi.configure(team=team)
            runs[team] = gi.align(rd.bases, rd.offsets, max_dist_per_read=dpr, **w.params())
            if team == 2:
                assert gi.last_call_stats()["wave_classes"] >= 1
    finally:
        gi.configure(team=-1)
    ref, ost = oracle.Index(g, w.seed_len).align(rd.bases, rd.offsets, max_dist_per_read=dpr,
                                                 threads=16, **w.params())
    assert_same(runs[2], ref, f"wave mode vs oracle ({case})")
    assert_same(runs[0], ref, f"warp mode vs oracle ({case})")
    assert_same(runs[1], ref, f"team mode vs oracle ({case})")
    if case == "exact_copies":
        assert ost.n_multiple > 20, ost.n_multiple
    else:
        assert ost.n_single > 200, ost.n_single
