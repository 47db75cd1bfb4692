#!/usr/bin/env python3
"""Benchmark of the SNAP alignment hot path on GB300.

One step = one alignment batch of the workload's reads (1M x 100 bp for the default
repeat-rich 100 Mbp workload) through the whole path: batch statistics, read
packing, seed probes, voting, bounded edit distances, hit selection.  The index is
built once before timing (its build time is reported separately, as the paper
times alignment separately from index construction).

value: reads/s with the reads already resident in HBM (CUDA events on the launch
stream, L2 flushed between steps).  e2e: the same metric through snap_align with
pinned host buffers (host-to-device copy of the reads and device-to-host copy of
the results inside the timed region).  roofline: the main align kernel's
algorithmic bytes (from the kernel's own counters) over its event-timed duration,
against the measured HBM copy bandwidth.  cpu_baseline: the CPU oracle on a bounded
sample of the same reads, all host cores, whose results are also compared with the
GPU's (parity_sample).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (replicas; each rank aligns its own reads against its own copy of the
index, no collective on the data path) runs under torch.distributed.run.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "reads/s aligned on 1 GB300 (bit-exact vs oracle) vs plain form; p50/p99 latency"
L2_FLUSH_BYTES = 512 << 20
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal (the measured copy peak is the denominator)


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="C2")
    ap.add_argument("--form", choices=["batched", "plain"], default="batched")
    ap.add_argument("--reads", type=int, default=0, help="override reads per step")
    ap.add_argument("--genome-bp", type=int, default=0,
                    help="scale the workload's genome to this many bases (same recipe), for "
                         "profiling a kernel on a small case")
    ap.add_argument("--batch", type=int, default=4_000_000,
                    help="reads per align call; a step aligns all the workload's reads")
    ap.add_argument("--serve", action="store_true",
                    help="serving run (C4 recipe): Poisson arrivals at --load x the measured "
                         "capacity, p50/p99 request latency")
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--serve-requests", type=int, default=200,
                    help="requests of the bounded serving pass in the default run (0: none)")
    ap.add_argument("--load", type=float, default=0.7)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--sweep-hmax", default="",
                    help="comma-separated h_max values: for each, reads/s of the batched form "
                         "and accuracy against the generator's truth (aligned %%, error %%)")
    ap.add_argument("--sweep-first-seeds", default="",
                    help="comma-separated first_seeds values (1 = Algorithm 1): the "
                         "seeds-first variant's reads/s and accuracy, as --sweep-hmax")
    ap.add_argument("--stride", type=int, default=1,
                    help="stride-k index: index windows at multiples of k, probe each seed "
                         "at k offsets (1 = every window, the default)")
    ap.add_argument("--calls-per-step", type=int, default=0,
                    help="align calls per timed step over the workload's reads (0 = enough "
                         "for --min-timed-s of timed work, so the clock record has several "
                         "samples); consecutive calls alternate between two device copies "
                         "of the reads")
    ap.add_argument("--min-timed-s", type=float, default=1.5)
    ap.add_argument("--sweep-gather", action="store_true",
                    help="the random-gather ceiling over chunk sizes, chunks in flight per "
                         "thread and threads per SM (one JSON line)")
    ap.add_argument("--collapse", action="store_true",
                    help="exact-duplicate collapsing in the parallel drain "
                         "(snap_params.collapse_duplicates = 1)")
    ap.add_argument("--divergence", type=float, default=None,
                    help="divergence of repeat copies (default: the recipe's 2%%)")
    ap.add_argument("--profile", action="store_true",
                    help="warm-up plus the timed steps only (no plain form, e2e or CPU "
                         "baseline): the command to run under ncu")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.profile:
        args.no_plain = args.no_cpu_baseline = True
        args.e2e_steps = 0
        args.serve_requests = 0
        args.calls_per_step = args.calls_per_step or 1
    return args


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def job_throughput(total_s: float, reads_per_rank: int, steps: int, ws: int, device=None):
    """Whole-job reads/s of N replicas (reads are independent; each rank aligns its own
    reads with its own index copy, no collective on the data path): every rank's
    timed seconds are reduced to the slowest rank's, and all ranks' reads count.
    Returns (reads/s, the slowest rank's seconds)."""
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total_s], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    return reads_per_rank * ws * steps / total_s, total_s


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _strip_comments(src: str) -> str:
    """C/C++ source without comments and blank runs (string and char literals kept)."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            while i < n and src[i] != "\n":
                i += 1
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def _kernel_source_hash():
    """Hash of the kernel sources' code (comments and layout ignored): a committed ncu
    capture stays valid across comment edits, and no longer once any code changed."""
    h = hashlib.sha256()
    cs = os.path.join(ROOT, "paper_1111_5572_gb300", "csrc")
    for fn in sorted(os.listdir(cs)):
        with open(os.path.join(cs, fn), encoding="utf-8") as f:
            h.update(fn.encode() + b"\0" + _strip_comments(f.read()).encode())
    return h.hexdigest()[:16]


def _ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` from a committed ncu summary, if taken on
    these kernel sources and this workload."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        ent = d.get(kernel)
        if (ent and ent.get("source_hash") == _kernel_source_hash() and
                ent.get("workload") == workload):
            return ent
    except Exception:
        pass
    return None


GATHER_ILP = (4, 8, 16)
GATHER_THREADS_PER_SM = (1024, 1536, 2048)


def gather_ceiling(snap, chunks=(32, 64), ilps=GATHER_ILP, tps=GATHER_THREADS_PER_SM):
    """The random-gather ceiling: the best GB/s of independent random reads of one
    aligned chunk over a sweep of chunks in flight per thread and threads per SM
    (8 GiB buffer, 2^28 reads per point)."""
    out = {}
    for cb in chunks:
        pts = [{"ilp": i, "threads_per_sm": t,
                "gbs": snap.measure_gather_config(8 << 30, cb, 1 << 28, i, t)}
               for i in ilps for t in tps]
        best = max(pts, key=lambda q: q["gbs"])
        out[f"chunk{cb}_gbs"] = best["gbs"]
        out[f"chunk{cb}_best_shape"] = {"ilp": best["ilp"],
                                        "threads_per_sm": best["threads_per_sm"]}
        out[f"chunk{cb}_sweep_min_gbs"] = min(q["gbs"] for q in pts)
    out["sweep"] = {"ilp": list(ilps), "threads_per_sm": list(tps)}
    return out


def run_gather_sweep(args):
    """--sweep-gather: the random-gather ceiling over chunk sizes 16-128 bytes,
    1-16 chunks in flight per thread and 256-2048 threads per SM; one JSON line."""
    import torch

    import paper_1111_5572_gb300 as snap
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    points = []
    with ClockSampler(0) as clk:
        for cb in (16, 32, 64, 128):
            for i in (1, 2, 4, 8, 16):
                for t in (256, 512, 1024, 1536, 2048):
                    g = snap.measure_gather_config(8 << 30, cb, 1 << 28, i, t)
                    points.append({"chunk_bytes": cb, "ilp": i, "threads_per_sm": t,
                                   "gbs": g, "g_reads_per_s": g / cb})
    best = {cb: max((q for q in points if q["chunk_bytes"] == cb), key=lambda q: q["gbs"])
            for cb in (16, 32, 64, 128)}
    peak, peak_kind = _peaks()
    line = {"mode": "sweep_gather", "unit": "GB/s", "buffer_bytes": 8 << 30,
            "reads_per_point": 1 << 28, "peak_copy_gbs": peak, "peak_kind": peak_kind,
            "best": {str(cb): q for cb, q in best.items()}, "points": points,
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def make_workload(args, rank: int):
    import synth
    w = synth.CONFIGS[args.workload]
    n = args.reads or w.n_reads
    if n <= 0:
        raise SystemExit(f"{args.workload} is a serving recipe: give --reads (or use --serve)")
    if args.genome_bp:
        w = w.scaled(G=args.genome_bp, n_reads=n)
    t0 = time.perf_counter()
    if args.divergence is None:
        g, _ = w.make_genome()
    else:
        g, _ = synth.genome(w.G, w.repeat_frac, divergence=args.divergence)
        w = w.scaled(G=w.G, n_reads=n, name=f"{w.name}-divergence-{args.divergence:g}")
    rd = w.make_reads(g, n=n, first_index=rank * n)
    dpr = w.max_dist_per_read(rd.lengths())
    return w, g, rd, dpr, time.perf_counter() - t0


def cpu_oracle_sample(w, g, rd, dpr, target_s: float = 12.0, max_reads: int = 400_000,
                      stride: int = 1):
    """Time the oracle (as it stands) on a bounded sample on all host cores."""
    import oracle
    cores = os.cpu_count() or 1
    restricted = w.G > 500_000_000
    if restricted:
        # a full sorted index of a 3.1 Gbp genome takes minutes and ~50 GB; the
        # oracle then indexes only the seeds of the sampled reads (same results)
        max_reads = min(max_reads, 100_000)
        cand = rd.subset(np.arange(min(rd.n, max_reads)))
        idx = oracle.Index(g, w.seed_len, kmer_filter=oracle.read_seed_kmers(
            cand.bases, cand.offsets, w.seed_len, w.num_seeds, stride), stride=stride)
    else:
        idx = oracle.Index(g, w.seed_len, stride=stride)
    probe = rd.subset(np.arange(min(rd.n, 20_000)))
    pd = None if dpr is None else dpr[:probe.n]
    t0 = time.perf_counter()
    idx.align(probe.bases, probe.offsets, max_dist_per_read=pd, threads=cores, **w.params())
    rate = probe.n / max(1e-6, time.perf_counter() - t0)
    n = int(min(rd.n, max_reads, max(probe.n, rate * target_s)))
    sample = np.arange(n)
    sub = rd.subset(sample) if n < rd.n else rd
    sd = None if dpr is None else dpr[:n]
    t0 = time.perf_counter()
    res, _ = idx.align(sub.bases, sub.offsets, max_dist_per_read=sd, threads=cores,
                       **w.params())
    dt = time.perf_counter() - t0
    # the same oracle on one core, on the first reads of the sample (about 2 s)
    one = rd.subset(np.arange(min(n, max(200, int(2.0 * rate / cores)))))
    t1 = time.perf_counter()
    idx.align(one.bases, one.offsets, max_dist_per_read=None if dpr is None else dpr[:one.n],
              threads=1, **w.params())
    one_rate = one.n / max(1e-6, time.perf_counter() - t1)
    what = ("index restricted to the sampled reads' seeds" if restricted
            else "index over the full genome")
    return dict(value=n / dt, unit="reads/s", cores=cores, kind="oracle",
                sample=f"first {n} reads of the workload, {what} "
                       f"(built in {idx.build_seconds:.1f} s, not timed)",
                single_core={"value": one_rate, "reads": one.n}), sample, res


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    w, g, rd, dpr, _ = make_workload(args, 0)
    cores = os.cpu_count() or 1
    idx = oracle.Index(g, w.seed_len, stride=args.stride)
    per_step = min(rd.n, 10_000)

    def step(k):
        lo = (k * per_step) % max(1, rd.n - per_step + 1)
        sub = rd.subset(np.arange(lo, lo + per_step))
        sd = None if dpr is None else dpr[lo:lo + per_step]
        idx.align(sub.bases, sub.offsets, max_dist_per_read=sd, threads=cores, **w.params())

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(args.warmup + k)
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "reads/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": w.name, "reads_per_step": per_step, "genome_bp": w.G,
                   "form": "cpu-oracle"},
        "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": "reads/s",
                         "sample": f"{per_step} reads per step, cycling through the "
                                   f"workload's {rd.n} reads"},
        "e2e": {"value": value, "unit": "reads/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1111_5572_gb300 as snap
    import __graft_entry__

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    __graft_entry__.build()

    w, g, rd, dpr, gen_s = make_workload(args, rank)
    n = rd.n
    t0 = time.perf_counter()
    idx = snap.Index(g, w.seed_len, stride=args.stride)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    info = idx.info()
    params = w.params()
    if args.collapse:
        params["collapse_duplicates"] = 1
    plain = args.form == "plain"

    d_b = torch.from_numpy(rd.bases).to(dev)
    d_o = torch.from_numpy(rd.offsets.view(np.int64)).to(dev)
    d_out = torch.zeros((n, 16), dtype=torch.uint8, device=dev)
    d_dpr = None if dpr is None else torch.from_numpy(dpr).to(dev)
    # a second device copy of the reads and results: consecutive calls of a step
    # alternate between the two, so a call never finds the previous call's reads
    # in L2 (the index itself is far larger than L2)
    copies = [(d_b, d_out), (d_b.clone(), torch.zeros_like(d_out))]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    # a stream of its own (not the legacy default stream) so the batched form can
    # replay its launch sequence as a CUDA graph
    stream = torch.cuda.Stream(device=dev)

    batch = max(1, min(args.batch, n))

    def one_pass(form_plain, which=0):
        # all the workload's reads, `batch` reads per call; returns each call's stats
        db, dout = copies[which]
        calls = []
        for b0 in range(0, n, batch):
            nb = min(batch, n - b0)
            idx.align_device(db, d_o[b0:b0 + nb + 1], dout[b0:b0 + nb],
                             d_max_dist_per_read=None if d_dpr is None else d_dpr[b0:b0 + nb],
                             stream=stream, plain=form_plain, **params)
            calls.append(idx.last_call_stats())
        return calls

    def flush_l2():
        # ordered before the step's first event; the read pass leaves L2 holding clean
        # lines, so the write-back of the zeroed buffer is not paid inside the step
        with torch.cuda.stream(stream):
            flush.zero_()
            flush.amax()

    def pass_ms(form_plain, reps=3):
        # device time of one pass over the workload (to size the timed steps)
        best = 1e30
        for k in range(reps):
            flush_l2()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one_pass(form_plain, k & 1)
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    def timed(form_plain, steps, warmup, passes):
        for k in range(warmup):
            flush_l2()
            one_pass(form_plain, k & 1)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        calls = []
        wall0 = time.perf_counter()
        with ClockSampler(local) as clk:
            for k in range(steps):
                flush_l2()  # L2 flush on the timed stream, before the step's first event
                evs[k][0].record(stream)
                step_calls = []
                for q in range(passes):
                    step_calls += one_pass(form_plain, q & 1)
                evs[k][1].record(stream)
                calls = step_calls
            torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        step_ms = [a.elapsed_time(b) for a, b in evs]
        return step_ms, calls, clk.summary(), wall

    for k in range(args.warmup):  # warm-up (tuning, graphs) before sizing the steps
        one_pass(plain, k & 1)
    passes = args.calls_per_step
    if passes <= 0:
        t_pass = pass_ms(plain) / 1e3
        passes = int(max(1, min(1000, np.ceil(args.min_timed_s / (args.steps * t_pass)))))
    step_ms, calls, clocks, wall = timed(plain, args.steps, args.warmup, passes)
    reads_per_step = n * passes
    value, total_s = job_throughput(sum(step_ms) / 1e3, reads_per_step, args.steps, ws, dev)
    ms_per_step = total_s * 1e3 / args.steps
    # every kernel launch of the last step's calls (stats, pack and align kernels)
    launches = int(sum(c["kernel_launches"] for c in calls)) * args.steps
    got = d_out.cpu().numpy().view(snap.RESULT_DTYPE).reshape(-1)

    # Roofline of the dominant kernel: algorithmic bytes per the survey's per-unit
    # figures (read in 100 B of bases at m = 100, i.e. m bytes, + 16 B result per read
    # finished; 32 B per probe; 4 B per out-of-line list entry; 64 B per scored
    # candidate) over the kernel's event-timed duration on the launch stream.
    mean_m = float(rd.lengths().mean())
    peak, peak_kind = _peaks()
    nc = len(calls)
    mean = lambda key: float(np.mean([c[key] for c in calls]))
    first = calls[0]  # counters of one call (every call aligns the same reads)
    pc = [c for c in calls[:max(1, len(calls) // passes)]]  # the calls of one pass
    tot = lambda key: float(sum(c[key] for c in pc))

    def alg_bytes(reads, probes, lists, eds):
        return reads * (mean_m + 16) + 32 * probes + 4 * lists + 64 * eds

    span_bytes = alg_bytes(tot("reads"), tot("seeds"), tot("list_entries"), tot("ed_calls"))
    span_ms = float(sum(c["align_ms"] for c in calls)) / passes
    light_ms = float(sum(c["light_ms"] for c in calls)) / passes
    light_bytes = alg_bytes(tot("reads_light"), tot("light_seeds"), tot("light_list_entries"),
                            tot("light_ed_calls"))
    if not plain and light_ms > 0.5 * span_ms:
        kname, kbytes, kms = "k_align_light", light_bytes, light_ms
    elif not plain:
        kname = "k_align_fused/k_align_team (per length class)"
        kbytes, kms = span_bytes - light_bytes, span_ms - light_ms
    else:
        kname, kbytes, kms = "plain stages", span_bytes, span_ms
    achieved = kbytes / (kms / 1e3) / 1e9
    tr = _ncu_traffic(kname.split(" ")[0].split("/")[0], w.name)
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_kind": f"{peak_kind} hbm_gbs",
                "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                # DRAM bytes of one launch from a committed ncu capture of this kernel's
                # current source on this workload (scaled to the call's read count)
                "traffic": None if tr is None else
                tr["dram_bytes_per_launch"] * tot("reads") / tr["reads"],
                "algorithmic_bytes_per_launch": kbytes, "kernel_ms": kms,
                "bytes_per_unit": {"read": f"{mean_m:.0f} + 16", "probe": 32, "list_entry": 4,
                                   "scored_candidate": 64},
                "align_span": {"kernels": "k_align_light + k_split_classes + "
                                          "k_align_fused/k_align_team per length class",
                               "algorithmic_bytes": span_bytes, "ms": span_ms,
                               "achieved": span_bytes / (span_ms / 1e3) / 1e9,
                               "frac": span_bytes / (span_ms / 1e3) / 1e9 / peak},
                "counters": {k: tot(k) for k in ("reads", "seeds", "slot_reads", "list_entries",
                                                 "ed_calls", "ed_over", "window_bytes",
                                                 "ed_filtered", "ed_collapsed", "reads_light", "light_seeds",
                                                 "light_list_entries", "light_ed_calls")}}
    # the practical ceiling of this traffic: independent random reads of one
    # aligned chunk (a 64-byte index bucket, a 32-byte sector); not under
    # --profile, whose launch list should hold the aligner's kernels only
    roofline["gather_ceiling"] = None
    if not args.profile:
        try:
            gc = gather_ceiling(snap)
            gc["frac_of_chunk64"] = achieved / gc["chunk64_gbs"]
            roofline["gather_ceiling"] = gc
        except Exception as e:  # a measurement aid, not the product
            roofline["gather_ceiling"] = {"error": str(e)[:200]}

    line = {
        "metric": METRIC, "value": value, "unit": "reads/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": w.name, "genome_bp": w.G, "repeat_frac": w.repeat_frac,
                   "reads_per_step": reads_per_step, "reads_per_call": batch,
                   "passes_per_step": passes,
                   "read_len": "100" if w.len_mode == 0 else "mixed",
                   "seed_len": w.seed_len, "index_stride": args.stride, **params,
                   "form": args.form,
                   "l2": "flushed before every step (512 MiB write, then a read of it, on the timed stream); "
                         "within a step, consecutive passes alternate between two device "
                         "copies of the reads",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "ms_per_pass": ms_per_step / passes,
        "bases_per_s": value * mean_m,
        "index_build_s": build_s, "index_device_gb": info["device_bytes"] / 1e9,
        "input_gen_s": gen_s, "wall_s_timed": wall,
        "gpu_launches": launches, "clocks": clocks, "roofline": roofline,
        "stage_ms_per_call": {k: mean(k) for k in ("stats_ms", "pack_ms", "align_ms",
                                                   "light_ms", "total_ms", "host_plan_ms")},
        "launch_shape": {k: first[k] for k in ("light_threads", "warps_per_block",
                                               "table_slots", "graph_replay", "team_classes")},
    }

    # the plain one-launch-per-stage form on the same GPU and inputs
    if not plain and not args.no_plain:
        try:
            p_ms, p_calls, _, _ = timed(True, max(3, args.steps // 4), 3, passes)
            p_got = d_out.cpu().numpy().view(snap.RESULT_DTYPE).reshape(-1)
            same = all(np.array_equal(p_got[f], got[f]) for f in
                       ("location", "edit_distance", "strand", "cls"))
            p_total = sum(p_ms) / 1e3
            line["plain"] = {"value": reads_per_step * len(p_ms) / p_total, "unit": "reads/s",
                             "ms_per_pass": p_total * 1e3 / len(p_ms) / passes,
                             "gpu_launches_per_call": int(p_calls[-1]["kernel_launches"]),
                             "identical_results": bool(same)}
            # the probe path alone: the plain form's seed-probe stage kernel, whose
            # traffic is the packed s-mer (8 B) and seed record (16 B) per seed, the
            # 16-byte index slots it reads, and per read its offsets and hit count
            ps = p_calls[-1]
            probe_ms = float(np.mean([q["probe_ms"] for q in p_calls]))
            probe_bytes = 24 * ps["seeds"] + 16 * ps["slot_reads"] + 20 * ps["reads"]
            if probe_ms > 0:
                gbs = probe_bytes / (probe_ms / 1e3) / 1e9
                line["probe_stage"] = {
                    "kernel": "k_plain_probe", "algorithmic_bytes": probe_bytes,
                    "kernel_ms": probe_ms, "achieved_gbs": gbs, "frac": gbs / peak,
                    "frac_of_nominal": gbs / NOMINAL_HBM_GBS,
                    "probes": ps["seeds"], "slot_reads": ps["slot_reads"],
                    "probes_per_s": ps["seeds"] / (probe_ms / 1e3)}
                gc = roofline.get("gather_ceiling") or {}
                if "chunk64_gbs" in gc:
                    line["probe_stage"]["frac_of_gather_chunk64"] = gbs / gc["chunk64_gbs"]
            line["batched_over_plain"] = line["value"] / line["plain"]["value"]
        except Exception as e:  # the plain form is a comparison, not the product
            line["plain"] = {"error": str(e)[:200]}

    # e2e through the public host-buffer call: pinned inputs in, results out
    if args.e2e_steps > 0:
        pin_b = torch.from_numpy(rd.bases).pin_memory()
        pin_o = torch.from_numpy(rd.offsets.view(np.int64)).pin_memory()
        pin_out = torch.zeros((n, 16), dtype=torch.uint8).pin_memory()
        nb, no = pin_b.numpy(), pin_o.numpy().view(np.uint64)
        no_out = pin_out.numpy().view(snap.RESULT_DTYPE).reshape(-1)
        def e2e_step():
            for b0 in range(0, n, batch):
                m_ = min(batch, n - b0)
                idx.align(nb, no[b0:b0 + m_ + 1],
                          max_dist_per_read=None if dpr is None else dpr[b0:b0 + m_],
                          out=no_out[b0:b0 + m_], plain=plain, **params)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        e2e_s = time.perf_counter() - t0
        line["e2e"] = {"value": n * args.e2e_steps / e2e_s, "unit": "reads/s",
                       "h2d_bytes_per_step": int(rd.bases.nbytes + rd.offsets.nbytes +
                                                 (0 if dpr is None else dpr.nbytes)),
                       "d2h_bytes_per_step": int(16 * n), "steps": args.e2e_steps}

    # a bounded serving pass: C4-recipe requests (100-1,000 reads each, 80% 100 bp and
    # 20% 1-10 kb at 5% error) on this workload's genome, p50/p99 latency at 0.7 x
    # the measured capacity, and the plain form on the same request stream
    if rank == 0 and args.serve_requests > 0 and not plain:
        import synth
        reqs = make_requests(g, synth.CONFIGS["C4"], args.serve_requests, 100, 1000,
                             first=10_000_000)
        sv = serving_pass(snap, idx, reqs, synth.CONFIGS["C4"].params(), args.load)
        sv["workload"] = (f"C4 recipe requests (log-uniform 100-1000 reads; 80% 100 bp, 20% "
                          f"1-10 kb at 5% error) on the {w.G // 1_000_000} Mbp genome")
        line["serving"] = sv

    if rank == 0 and not args.no_cpu_baseline:
        cb, sample, ref = cpu_oracle_sample(w, g, rd, dpr, stride=args.stride)
        line["cpu_baseline"] = cb
        mism = sum(int((got[f][sample] != ref[f]).sum()) for f in
                   ("location", "edit_distance", "strand", "cls"))
        line["parity_sample"] = {"reads": int(len(sample)), "field_mismatches": mism}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def make_requests(g, w, n_requests: int, lo: int, hi: int, first: int = 0):
    """Serving requests of the C4 recipe on genome g: request sizes log-uniform in
    [lo, hi] reads, each read 100 bp (80%) or log-uniform 1-10 kb (20%), 5% error,
    d_max = max(8, ceil(0.08 m)).  Returns [(reads, d_max per read)]."""
    import synth
    _, sizes = synth.arrivals(n_requests, 1.0, lo, hi)
    reqs = []
    for k, nr in enumerate(sizes.tolist()):
        lens = synth.read_lengths(nr, 2, 100, 1000, 10000, 0.8, seed=1000 + k)
        rd = synth.reads(g, lens, w.sub_rate, w.indel_rate, w.indel_len, first_index=first)
        first += nr
        reqs.append((rd, w.max_dist_per_read(rd.lengths())))
    return reqs


def serving_pass(snap, gi, reqs, params, load: float, max_inflight: int = 4,
                 plain_compare: bool = True, mem_budget_bytes: int = 64 << 30):
    """Serve `reqs` on index gi: first all at once (capacity), then submitted at
    Poisson arrival times at load x capacity; latency = completion - submission.
    With plain_compare, the same requests also go one at a time through the plain
    one-launch-per-stage form at the same arrival times (a request waits for the one
    before it).  Returns a dict of reads/s, capacity and p50/p99 latency."""
    import synth
    total_reads = int(sum(r.n for r, _ in reqs))
    total_bases = int(sum(int(r.offsets[-1]) for r, _ in reqs))
    srv = snap.Server(gi, mem_budget_bytes=mem_budget_bytes, max_inflight=max_inflight)
    try:
        for rd, dpr in reqs[:3]:  # warm-up (tuning, graphs)
            srv.wait(srv.submit(rd.bases, rd.offsets, max_dist_per_read=dpr, **params))
        t0 = time.perf_counter()
        tk = [srv.submit(rd.bases, rd.offsets, max_dist_per_read=dpr, **params)
              for rd, dpr in reqs]
        results = [srv.wait(t)[0] for t in tk]
        cap_s = time.perf_counter() - t0
        capacity = total_reads / cap_s
        rate = load * capacity / (total_reads / len(reqs))  # requests per second
        times, _ = synth.arrivals(len(reqs), rate, 1, 2)
        lat = [0.0] * len(reqs)
        tickets = [None] * len(reqs)
        start = time.perf_counter()
        for k, (rd, dpr) in enumerate(reqs):
            delay = start + float(times[k]) - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets[k] = srv.submit(rd.bases, rd.offsets, max_dist_per_read=dpr, **params)
        same = True
        for k in range(len(reqs)):
            res, lat[k] = srv.wait(tickets[k])
            same &= all(np.array_equal(res[f], results[k][f])
                        for f in ("location", "edit_distance", "strand", "cls"))
        wall = time.perf_counter() - start
    finally:
        srv.close()
    out = {"requests": len(reqs), "reads": total_reads, "bases": total_bases,
           "max_inflight": max_inflight, "offered_load": load, "arrival_rate_per_s": rate,
           "capacity_reads_per_s": capacity, "capacity_bases_per_s": total_bases / cap_s,
           "value_reads_per_s": total_reads / wall,
           "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
           "max_s": float(max(lat)), "results_same_alone_and_in_mix": bool(same)}
    if plain_compare:
        # the plain form on the same requests: capacity back to back, then the same
        # arrival times with one request on the device at a time
        for rd, dpr in reqs[:2]:
            gi.align(rd.bases, rd.offsets, max_dist_per_read=dpr, plain=True, **params)
        t0 = time.perf_counter()
        same_plain = True
        for k, (rd, dpr) in enumerate(reqs):
            res = gi.align(rd.bases, rd.offsets, max_dist_per_read=dpr, plain=True, **params)
            same_plain &= all(np.array_equal(res[f], results[k][f])
                              for f in ("location", "edit_distance", "strand", "cls"))
        p_cap = total_reads / (time.perf_counter() - t0)
        plat = []
        start = time.perf_counter()
        for k, (rd, dpr) in enumerate(reqs):
            arrive = start + float(times[k])
            delay = arrive - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            gi.align(rd.bases, rd.offsets, max_dist_per_read=dpr, plain=True, **params)
            plat.append(time.perf_counter() - arrive)
        p_wall = time.perf_counter() - start
        out["plain"] = {"capacity_reads_per_s": p_cap, "value_reads_per_s": total_reads / p_wall,
                        "p50_s": float(np.percentile(plat, 50)),
                        "p99_s": float(np.percentile(plat, 99)),
                        "identical_results": bool(same_plain)}
        out["served_over_plain_capacity"] = capacity / p_cap
    return out


def run_serve(args):
    """C4 serving run on the 3.1 Gbp genome: requests of log-uniform size (1k-100k
    reads; 80% 100 bp, 20% 1-10 kb), first all submitted at once to measure
    capacity, then submitted at Poisson arrival times at --load x capacity."""
    import torch

    import paper_1111_5572_gb300 as snap
    import synth
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    w = synth.CONFIGS["C4"]
    t0 = time.perf_counter()
    g, _ = w.make_genome()
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    gi = snap.Index(g, w.seed_len)
    build_s = time.perf_counter() - t0
    reqs = make_requests(g, w, args.requests, 1000, 100_000)
    with ClockSampler(0) as clk:
        sv = serving_pass(snap, gi, reqs, w.params(), args.load, plain_compare=False)
    line = {
        "metric": METRIC, "mode": "serve", "value": sv["value_reads_per_s"], "unit": "reads/s",
        "n_gpus": 1, "higher_is_better": True, "dtype": "u8", "data": "synthetic",
        "config": {"workload": w.name, "genome_bp": w.G, "request_reads": "log-uniform "
                   "[1000, 100000]", **{k: sv[k] for k in ("requests", "reads", "bases",
                                                          "max_inflight", "offered_load",
                                                          "arrival_rate_per_s")}},
        "capacity_reads_per_s": sv["capacity_reads_per_s"],
        "capacity_bases_per_s": sv["capacity_bases_per_s"],
        "latency_s": {"p50": sv["p50_s"], "p99": sv["p99_s"], "max": sv["max_s"]},
        "results_same_alone_and_in_mix": sv["results_same_alone_and_in_mix"],
        "index_build_s": build_s, "genome_gen_s": gen_s, "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


# A confident alignment is correct when it is on the read's true strand and within
# this many bases of its true start (the configs' longest indel is 20 bases).
CORRECT_WINDOW = 20


def accuracy(got, rd) -> dict:
    """Aligned % (single-hit class: the paper's confidently mapped reads) and error %
    (confident reads on the wrong strand or more than CORRECT_WINDOW bases away)."""
    cls = got["cls"].astype(np.int64)
    single = cls == 1
    ok = single & (got["strand"].astype(np.int64) == rd.strand.astype(np.int64)) & \
        (np.abs(got["location"].astype(np.int64) - rd.origin) <= CORRECT_WINDOW)
    ns = int(single.sum())
    return {"aligned_pct": 100.0 * ns / len(cls),
            "error_pct": 100.0 * (ns - int(ok.sum())) / max(1, ns),
            "multiple_pct": 100.0 * float((cls == 2).mean()),
            "not_found_pct": 100.0 * float((cls == 0).mean())}


def run_sweep(args, param: str, values):
    """Parameter sweep of the batched form: for each value of `param` (max_hits: the
    h_max trade-off of Ongoing Work, Observations; first_seeds: the seeds-first variant
    of Local Alignment), device-resident reads/s over the workload's reads, accuracy
    against the generator's truth, and a parity sample against the oracle."""
    import torch

    import oracle
    import paper_1111_5572_gb300 as snap
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    w, g, rd, dpr, gen_s = make_workload(args, 0)
    n = rd.n
    idx = snap.Index(g, w.seed_len, stride=args.stride)
    d_b = torch.from_numpy(rd.bases).to(dev)
    d_o = torch.from_numpy(rd.offsets.view(np.int64)).to(dev)
    d_out = torch.zeros((n, 16), dtype=torch.uint8, device=dev)
    d_dpr = None if dpr is None else torch.from_numpy(dpr).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    batch = max(1, min(args.batch, n))
    sample = rd.subset(np.arange(min(n, 20_000)))
    restricted = w.G > 500_000_000
    oidx = oracle.Index(g, w.seed_len, kmer_filter=oracle.read_seed_kmers(
        sample.bases, sample.offsets, w.seed_len, w.num_seeds, args.stride)
        if restricted else None, stride=args.stride)
    points = []
    with ClockSampler(0) as clk:
        for h in values:
            params = dict(w.params(), **{param: h})

            def step():
                for b0 in range(0, n, batch):
                    m_ = min(batch, n - b0)
                    idx.align_device(d_b, d_o[b0:b0 + m_ + 1], d_out[b0:b0 + m_],
                                     d_max_dist_per_read=None if d_dpr is None
                                     else d_dpr[b0:b0 + m_], stream=stream, **params)

            for _ in range(max(3, args.warmup)):
                step()
            torch.cuda.synchronize()
            ms = []
            for _ in range(args.steps):
                with torch.cuda.stream(stream):  # before the step's first event, as above
                    flush.zero_()
                    flush.amax()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step()
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            got = d_out.cpu().numpy().view(snap.RESULT_DTYPE).reshape(-1)
            ref, _ = oidx.align(sample.bases, sample.offsets,
                                max_dist_per_read=None if dpr is None else dpr[:sample.n],
                                threads=os.cpu_count() or 1, **params)
            mism = sum(int((got[f][:sample.n] != ref[f]).sum())
                       for f in ("location", "edit_distance", "strand", "cls"))
            points.append({param: h, "reads_per_s": n * len(ms) / (sum(ms) / 1e3),
                           "ms_per_step": sum(ms) / len(ms), **accuracy(got, rd),
                           "parity_sample": {"reads": sample.n, "field_mismatches": mism}})
    line = {"metric": METRIC, "mode": f"sweep_{param}", "unit": "reads/s", "n_gpus": 1,
            "dtype": "u8", "data": "synthetic",
            "config": {"workload": w.name, "genome_bp": w.G, "reads": n, "index_stride": args.stride,
                       "correct_window_bases": CORRECT_WINDOW, "steps": args.steps,
                       "l2": "flushed between steps (512 MiB write, then a read of it)"},
            "points": points, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    if args.serve:
        return run_serve(args)
    if args.sweep_gather:
        return run_gather_sweep(args)
    if args.sweep_hmax:
        return run_sweep(args, "max_hits", [int(x) for x in args.sweep_hmax.split(",") if x])
    if args.sweep_first_seeds:
        return run_sweep(args, "first_seeds",
                         [int(x) for x in args.sweep_first_seeds.split(",") if x])
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
