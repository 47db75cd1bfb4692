"""The allocation-free entry point, snap_align_device_noalloc.

It is meant for callers that cannot let the library allocate device memory: code
under a framework that already owns the device memory pool, serving threads that
must not stall the device with cudaMalloc/cudaFree, or processes that route every
device allocation through their own allocator.  Its scratch is one fixed array
inside the library, so these tests check that it gives exactly the results of
snap_align_device on two calls in a row (the array keeps the previous call's
contents), including reads whose candidate tables outgrow shared memory and are
aligned by its second launch; that a call changes the device's free memory by
nothing; that batches beyond the array's limits are refused with a clear error;
and that on the 1M-read benchmark batch it stays within a small factor of
snap_align_device's time.

This file is collected last so that a failure here does not hide any other test.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

FIELDS = ("location", "edit_distance", "strand", "cls")


@pytest.fixture(scope="module")
def snap():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1111_5572_gb300 as m
    return m


def _device_batch(rd, dev):
    import torch
    d_b = torch.from_numpy(rd.bases).to(dev)
    d_o = torch.from_numpy(rd.offsets.view(np.int64)).to(dev)
    return d_b, d_o


def test_noalloc_matches_allocating_entry_point_twice(snap):
    import torch
    dev = torch.device("cuda:0")
    # repeat-rich genome, 100 bp and long reads: exercises the shared-memory and the
    # in-array candidate tables and the long-read edit distance
    w = synth.CONFIGS["C2"].scaled(G=3_000_000, n_reads=20_000)
    g, _ = w.make_genome()
    rd = w.make_reads(g)
    idx = snap.Index(g, w.seed_len)
    d_b, d_o = _device_batch(rd, dev)
    stream = torch.cuda.current_stream()
    ref = torch.zeros((rd.n, 16), dtype=torch.uint8, device=dev)
    idx.align_device(d_b, d_o, ref, stream=stream, **w.params())
    ref_np = ref.cpu().numpy().view(snap.RESULT_DTYPE).reshape(-1)
    for call in range(2):
        out = torch.full((rd.n, 16), 0xAB, dtype=torch.uint8, device=dev)
        torch.cuda.synchronize()
        free_before, _ = torch.cuda.mem_get_info()
        idx.align_device_noalloc(d_b, d_o, out, stream=stream, **w.params())
        torch.cuda.synchronize()
        free_after, _ = torch.cuda.mem_get_info()
        got = out.cpu().numpy().view(snap.RESULT_DTYPE).reshape(-1)
        for f in FIELDS:
            assert np.array_equal(got[f], ref_np[f]), f"call {call}: field {f} differs"
        if call == 1:  # the array exists once the library's code is on the device
            assert free_after == free_before

    # uneven lengths with per-read limits (long reads take the shared-memory diagonals)
    w4 = synth.CONFIGS["C4"].scaled(G=2_000_000, n_reads=200)
    g4, _ = w4.make_genome()
    rd4 = w4.make_reads(g4, n=200)
    dpr = torch.from_numpy(w4.max_dist_per_read(rd4.lengths())).to(dev)
    idx4 = snap.Index(g4, w4.seed_len)
    d_b4, d_o4 = _device_batch(rd4, dev)
    ref4 = torch.zeros((rd4.n, 16), dtype=torch.uint8, device=dev)
    idx4.align_device(d_b4, d_o4, ref4, d_max_dist_per_read=dpr, stream=stream, **w4.params())
    for _ in range(2):
        out4 = torch.zeros((rd4.n, 16), dtype=torch.uint8, device=dev)
        idx4.align_device_noalloc(d_b4, d_o4, out4, d_max_dist_per_read=dpr, stream=stream,
                                  **w4.params())
        assert torch.equal(out4, ref4)


def test_noalloc_refuses_batches_over_its_limit(snap):
    import torch
    dev = torch.device("cuda:0")
    g, _ = synth.genome(200_000, 0.0)
    idx = snap.Index(g, 20)
    n, m = 2_100_000, 100   # 210M bases > the 201M-base limit
    d_b = torch.full((n * m,), ord("A"), dtype=torch.uint8, device=dev)
    d_o = torch.arange(0, n * m + 1, m, dtype=torch.int64, device=dev)
    out = torch.zeros((n, 16), dtype=torch.uint8, device=dev)
    with pytest.raises(snap.SnapError) as e:
        idx.align_device_noalloc(d_b, d_o, out)
    assert e.value.code == snap.SNAP_E_INVAL
    assert "at most" in str(e.value)
    # the refusal leaves the entry point usable
    small = torch.full((1000,), ord("A"), dtype=torch.uint8, device=dev)
    small[:100] = torch.from_numpy(g[5000:5100]).to(dev)
    offs = torch.tensor([0, 100], dtype=torch.int64, device=dev)
    o1 = torch.zeros((1, 16), dtype=torch.uint8, device=dev)
    idx.align_device_noalloc(small, offs, o1)
    r = o1.cpu().numpy().view(snap.RESULT_DTYPE).reshape(-1)
    assert int(r["cls"][0]) == snap.SINGLE_HIT and int(r["location"][0]) == 5000


def _planted_repeat_batch(n_copies=400, unit=200, G=2_000_000, n=3000):
    """A random genome with one exact 200-base unit planted n_copies times, and reads
    half from unit copies (every seed hits n_copies places) and half elsewhere."""
    rng = np.random.default_rng(11)
    g = np.frombuffer(b"ACGT", dtype=np.uint8)[rng.integers(0, 4, G)].copy()
    u = g[1000:1000 + unit].copy()
    starts = np.sort(rng.choice(np.arange(10_000, G - unit, unit + 7), n_copies, replace=False))
    for p0 in starts:
        g[p0:p0 + unit] = u
    lens = np.full(n, 100, dtype=np.uint32)
    rd = synth.reads(g, lens, 0.01, 0.001, (1, 3), seed=21)
    # every other read taken from inside a copy of the unit
    for i in range(0, n, 2):
        p0 = int(starts[i % n_copies]) + (i % 90)
        rd.bases[rd.offsets[i]:rd.offsets[i + 1]] = g[p0:p0 + 100]
    return g, rd


def test_noalloc_second_launch_for_large_candidate_sets(snap):
    import torch
    dev = torch.device("cuda:0")
    g, rd = _planted_repeat_batch()
    idx = snap.Index(g, 20)
    params = dict(max_dist=8, max_hits=3000, conf_diff=2, num_seeds=5)
    d_b, d_o = _device_batch(rd, dev)
    ref = torch.zeros((rd.n, 16), dtype=torch.uint8, device=dev)
    # the unit's reads have 5 x 401 hits: more than the 256 a shared-memory table of
    # the allocation-free call holds, so they go through its second launch
    idx.align_device(d_b, d_o, ref, **params)
    for _ in range(2):
        out = torch.full((rd.n, 16), 0x5C, dtype=torch.uint8, device=dev)
        idx.align_device_noalloc(d_b, d_o, out, **params)
        assert torch.equal(out, ref)
    res = ref.cpu().numpy().view(snap.RESULT_DTYPE).reshape(-1)
    assert (res["cls"][0::2] == snap.MULTIPLE_HITS).mean() > 0.9  # the unit reads


def test_noalloc_refuses_candidate_tables_over_its_limit(snap):
    import torch
    dev = torch.device("cuda:0")
    g, _ = synth.genome(200_000, 0.0)
    idx = snap.Index(g, 20)
    # 1000 seeds x max_hits 300 = 300,000 > the 262,144 one warp's table may hold
    m = 20_000
    d_b = torch.from_numpy(np.tile(g[:m // 10], 10)).to(dev)
    d_o = torch.tensor([0, m], dtype=torch.int64, device=dev)
    out = torch.zeros((1, 16), dtype=torch.uint8, device=dev)
    with pytest.raises(snap.SnapError) as e:
        idx.align_device_noalloc(d_b, d_o, out, max_dist=8, max_hits=300, num_seeds=1000)
    assert e.value.code == snap.SNAP_E_INVAL
    assert "candidate table" in str(e.value)
    idx.align_device(d_b, d_o, out, max_dist=8, max_hits=300, num_seeds=1000)  # accepted there


def test_noalloc_time_on_the_benchmark_batch(snap):
    import torch
    dev = torch.device("cuda:0")
    w = synth.CONFIGS["C2"]
    g, _ = w.make_genome()
    rd = w.make_reads(g)
    idx = snap.Index(g, w.seed_len)
    d_b, d_o = _device_batch(rd, dev)
    out = torch.zeros((rd.n, 16), dtype=torch.uint8, device=dev)
    ref = torch.zeros((rd.n, 16), dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def best_ms(call, k=3):
        ms = []
        for _ in range(k):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            call()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return min(ms)

    alloc = lambda: idx.align_device(d_b, d_o, ref, stream=stream, **w.params())
    noalloc = lambda: idx.align_device_noalloc(d_b, d_o, out, stream=stream, **w.params())
    alloc()
    noalloc()
    t_alloc, t_noalloc = best_ms(alloc), best_ms(noalloc)
    assert torch.equal(out, ref)
    # one warp per read instead of the thread-per-read bucket, but every SM busy
    assert t_noalloc < 6.0 * t_alloc, (t_noalloc, t_alloc)

