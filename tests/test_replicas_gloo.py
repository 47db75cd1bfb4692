"""The multi-GPU path is replicas (reads are independent, Multi-Core Implementation):
each rank aligns its own reads with its own index copy and the only cross-rank step is
the timing reduction.  Checked here on CPU with two gloo ranks: the job's reads/s counts
every rank's reads over the slowest rank's time, and the ranks' read batches are
disjoint slices of one seeded stream."""
import os
import socket
import sys

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    sys.path.insert(0, ROOT)
    import bench
    # rank 1 is the slow one: 3 s against 2 s for 1000 reads x 5 steps each
    value, slowest = bench.job_throughput(2.0 + rank, 1000, 5, ws)
    q.put((rank, value, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_job_throughput_over_two_gloo_ranks():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, slowest in got:
        assert slowest == 3.0
        assert np.isclose(value, 2 * 1000 * 5 / 3.0)


def test_single_rank_needs_no_process_group():
    import bench
    value, t = bench.job_throughput(2.0, 1000, 5, 1)
    assert t == 2.0 and np.isclose(value, 2500.0)


def test_replica_reads_are_disjoint_slices_of_one_stream():
    import synth
    w = synth.CONFIGS["C1"].scaled(G=200_000, n_reads=0)
    g, _ = w.make_genome()
    n = 500
    r0 = w.make_reads(g, n=n, first_index=0)
    r1 = w.make_reads(g, n=n, first_index=n)
    both = w.make_reads(g, n=2 * n, first_index=0)
    assert np.array_equal(np.concatenate([r0.origin, r1.origin]), both.origin)
    assert np.array_equal(np.concatenate([r0.bases, r1.bases]), both.bases)
