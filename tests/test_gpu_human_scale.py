"""Human-scale workloads on the 3.1 Gbp synthetic genome (50% repeat families).

C5: 100M x 100 bp reads aligned in 4M-read batches with the batched form, the way
bench.py --workload C5 runs them; 20,000 reads sampled across all batches are
checked field by field against the oracle (its index restricted to the seeds those
reads look up), and every read is checked for properties that hold at any size.
C4: a sample of the serving recipe's mixed requests (80% 100 bp, 20% 1-10 kb at
5% error, d_max = max(8, ceil(0.08 m))) against the full genome, served through
the serving loop and checked against the oracle.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

FIELDS = ("location", "edit_distance", "strand", "cls")
C5_BATCH = 4_000_000


@pytest.fixture(scope="module")
def human():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1111_5572_gb300 as snap
    w = synth.CONFIGS["C5"]
    g, _ = w.make_genome()
    gi = snap.Index(g, w.seed_len)
    yield snap, g, gi
    gi.close()
    torch.cuda.empty_cache()


def _assert_same(got, ref, what):
    for f in FIELDS:
        if not np.array_equal(got[f], ref[f]):
            bad = np.nonzero(got[f] != ref[f])[0]
            raise AssertionError(f"{what}: {f} differs at {len(bad)} of {len(ref)} reads")


def test_c5_100M_reads_sampled(human):
    import torch
    snap, g, gi = human
    w = synth.CONFIGS["C5"]
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(5)
    n_total = w.n_reads
    sample = np.sort(rng.choice(n_total, 20_000, replace=False))
    got_sample = np.zeros(len(sample), dtype=snap.RESULT_DTYPE)
    counts = np.zeros(3, dtype=np.int64)
    for b0 in range(0, n_total, C5_BATCH):
        n = min(C5_BATCH, n_total - b0)
        rd = w.make_reads(g, n=n, first_index=b0)
        d_b = torch.from_numpy(rd.bases).to(dev)
        d_o = torch.from_numpy(rd.offsets.view(np.int64)).to(dev)
        out = torch.zeros((n, 16), dtype=torch.uint8, device=dev)
        gi.align_device(d_b, d_o, out, stream=stream, **w.params())
        res = out.cpu().numpy().view(snap.RESULT_DTYPE).reshape(-1)
        loc = res["location"] >= 0
        assert set(np.unique(res["cls"]).tolist()) <= {0, 1, 2}
        assert (res["edit_distance"][loc] <= w.max_dist).all()
        assert (res["edit_distance"][loc] >= 0).all()
        assert (res["location"][loc] < w.G).all()
        assert ((res["location"] == -1) == (res["edit_distance"] == -1)).all()
        assert (res["cls"][~loc] != snap.SINGLE_HIT).all()
        counts += np.bincount(res["cls"], minlength=3)
        sel = (sample >= b0) & (sample < b0 + n)
        got_sample[sel] = res[sample[sel] - b0]
    assert counts.sum() == n_total
    # oracle on the sampled reads (regenerated from their own streams)
    lens = np.full(len(sample), 100, dtype=np.uint32)
    sub_bases, offs = [], [0]
    for i in sample:
        one = synth.reads(g, lens[:1], w.sub_rate, w.indel_rate, w.indel_len,
                          first_index=int(i), threads=1)
        sub_bases.append(one.bases)
        offs.append(offs[-1] + one.bases.shape[0])
    bases = np.concatenate(sub_bases)
    offs = np.array(offs, dtype=np.uint64)
    keys = oracle.read_seed_kmers(bases, offs, w.seed_len, w.num_seeds)
    oi = oracle.Index(g, w.seed_len, kmer_filter=keys)
    ref, st = oi.align(bases, offs, threads=8, **w.params())
    _assert_same(got_sample, ref, "C5 sample")
    assert counts[snap.SINGLE_HIT] > 0.6 * n_total


def test_c4_mixed_requests_full_genome(human):
    snap, g, gi = human
    w = synth.CONFIGS["C4"]
    rng = np.random.default_rng(6)
    srv = snap.Server(gi, mem_budget_bytes=16 << 30, max_inflight=4)
    reqs, tickets = [], []
    first = 0
    for k, n in enumerate((3000, 1000, 5000, 1500)):
        lens = synth.read_lengths(n, 2, 100, 1000, 10000, 0.8, seed=500 + k)
        rd = synth.reads(g, lens, w.sub_rate, w.indel_rate, w.indel_len, first_index=first)
        first += n
        dpr = w.max_dist_per_read(rd.lengths())
        reqs.append((rd, dpr))
        tickets.append(srv.submit(rd.bases, rd.offsets, max_dist_per_read=dpr, **w.params()))
    results = [srv.wait(t)[0] for t in tickets]
    srv.close()
    # oracle on every short read of request 1 and 40 long reads across requests
    rd, dpr = reqs[1]
    keys = oracle.read_seed_kmers(rd.bases, rd.offsets, w.seed_len, w.num_seeds)
    ref, _ = oracle.Index(g, w.seed_len, kmer_filter=keys).align(
        rd.bases, rd.offsets, max_dist_per_read=dpr, threads=8, **w.params())
    _assert_same(results[1], ref, "C4 request 1")
    picks = []
    for k, (rd, dpr) in enumerate(reqs):
        long_ids = np.nonzero(rd.lengths() >= 1000)[0]
        for i in rng.choice(long_ids, min(10, len(long_ids)), replace=False):
            picks.append((k, int(i)))
    sub_b, offs, dprs, got = [], [0], [], []
    for k, i in picks:
        rd, dpr = reqs[k]
        b = rd.bases[rd.offsets[i]:rd.offsets[i + 1]]
        sub_b.append(b)
        offs.append(offs[-1] + b.shape[0])
        dprs.append(dpr[i])
        got.append(results[k][i])
    bases = np.concatenate(sub_b)
    offs = np.array(offs, dtype=np.uint64)
    dprs = np.array(dprs, dtype=np.int32)
    keys = oracle.read_seed_kmers(bases, offs, w.seed_len, w.num_seeds)
    ref, _ = oracle.Index(g, w.seed_len, kmer_filter=keys).align(
        bases, offs, max_dist_per_read=dprs, threads=8, **w.params())
    _assert_same(np.array(got, dtype=snap.RESULT_DTYPE), ref, "C4 long reads")


@pytest.mark.parametrize("team", [0, 1, 2])
def test_long_reads_full_genome_warp_and_team(human, team):
    """320 reads of 1-10 kb (log-uniform) with the serving recipe's error model and
    limits (d_max = max(8, ceil(0.08 m)), up to 800) on the 3.1 Gbp genome, aligned
    with one warp per read (team=0), in team mode (team=1) and in wave mode (team=2),
    the last two for every long class, each checked field by field against the
    oracle."""
    snap, g, gi = human
    w = synth.CONFIGS["C4"]
    lens = synth.read_lengths(320, 1, 100, 1000, 10000, 0.0, seed=900)
    rd = synth.reads(g, lens, w.sub_rate, w.indel_rate, w.indel_len, first_index=20_000_000)
    dpr = w.max_dist_per_read(rd.lengths())
    assert rd.lengths().min() >= 1000 and dpr.max() > 400
    gi.configure(team=team)
    try:
        got = gi.align(rd.bases, rd.offsets, max_dist_per_read=dpr, **w.params())
        st = gi.last_call_stats()
    finally:
        gi.configure(team=-1)
    # every length class present has limits above 31, so team=1 puts each in team mode
    classes = {int(m > 256) + int(m > 1024) + int(m > 4096) for m in rd.lengths().tolist()}
    assert st["team_classes"] == (0 if team == 0 else len(classes)), st["team_classes"]
    assert st["wave_classes"] == (len(classes) if team == 2 else 0), st["wave_classes"]
    keys = oracle.read_seed_kmers(rd.bases, rd.offsets, w.seed_len, w.num_seeds)
    ref, ost = oracle.Index(g, w.seed_len, kmer_filter=keys).align(
        rd.bases, rd.offsets, max_dist_per_read=dpr, threads=16, **w.params())
    _assert_same(got, ref, f"long reads team={team}")
    assert ost.n_single > 100

