"""The serving loop: requests of mixed sizes and read lengths submitted together run
concurrently (several slots, each with its own stream), and every request's results
are the same as when it is aligned alone, and as the oracle's.  A request larger
than the memory budget fails with SNAP_E_NOMEM without disturbing the others."""
import threading

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


def _same(a, b):
    return all(np.array_equal(a[f], b[f]) for f in FIELDS)


def test_requests_alone_equal_requests_in_the_mix(snap):
    # C4 recipe, scaled: 80% 100 bp and 20% long reads, per-read d_max
    w = synth.CONFIGS["C4"].scaled(G=3_000_000, n_reads=0)
    g, _ = w.make_genome()
    gi = snap.Index(g, w.seed_len)
    rng = np.random.default_rng(4)
    sizes = [int(x) for x in rng.integers(200, 3000, 10)] + [20, 5000]
    reqs = []
    first = 0
    for k, n in enumerate(sizes):
        lens = synth.read_lengths(n, 2, 100, 1000, 3000, 0.8, seed=100 + k)
        rd = synth.reads(g, lens, w.sub_rate, w.indel_rate, w.indel_len, first_index=first)
        first += n
        reqs.append((rd, w.max_dist_per_read(rd.lengths())))
    alone = [gi.align(rd.bases, rd.offsets, max_dist_per_read=dpr, **w.params())
             for rd, dpr in reqs]
    srv = snap.Server(gi, mem_budget_bytes=8 << 30, max_inflight=4)
    tickets = [srv.submit(rd.bases, rd.offsets, max_dist_per_read=dpr, **w.params())
               for rd, dpr in reqs]
    lat = []
    for t, ref in zip(tickets, alone):
        got, l = srv.wait(t)
        assert _same(got, ref)
        lat.append(l)
    assert all(x > 0 for x in lat)
    # submissions from several threads at once, waits in reverse order
    out = {}

    def submitter(ks):
        for k in ks:
            rd, dpr = reqs[k]
            out[k] = srv.submit(rd.bases, rd.offsets, max_dist_per_read=dpr, **w.params())

    th = [threading.Thread(target=submitter, args=(range(i, len(reqs), 3),)) for i in range(3)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for k in sorted(out, reverse=True):
        got, _ = srv.wait(out[k])
        assert _same(got, alone[k]), k
    srv.close()
    # and the oracle agrees on one of the requests
    rd, dpr = reqs[3]
    ref, _ = oracle.Index(g, w.seed_len).align(rd.bases, rd.offsets, max_dist_per_read=dpr,
                                                threads=4, **w.params())
    assert _same(alone[3], ref)


def test_budget_admission_and_refusal(snap):
    w = synth.CONFIGS["C1"].scaled(G=500_000, n_reads=4000)
    g, _ = w.make_genome()
    gi = snap.Index(g, w.seed_len)
    small = w.make_reads(g, n=2000)
    big = w.make_reads(g, n=200_000, first_index=10_000)
    ref_small = gi.align(small.bases, small.offsets, **w.params())
    # budget for one small request at a time (each request is charged its data plus
    # the slot's 256 MiB candidate-table allowance): requests queue and are admitted
    # in arrival order as memory frees up; the big one can never fit
    srv = snap.Server(gi, mem_budget_bytes=270 << 20, max_inflight=4)
    t1 = srv.submit(small.bases, small.offsets, **w.params())
    t2 = srv.submit(big.bases, big.offsets, **w.params())
    t3 = srv.submit(small.bases, small.offsets, **w.params())
    got1, _ = srv.wait(t1)
    with pytest.raises(snap.SnapError) as e:
        srv.wait(t2)
    assert e.value.code == snap.SNAP_E_NOMEM
    got3, _ = srv.wait(t3)
    assert _same(got1, ref_small) and _same(got3, ref_small)
    srv.close()
    with pytest.raises(snap.SnapError):
        snap.Server(gi, mem_budget_bytes=1 << 30, max_inflight=0)
