"""Seeded synthetic inputs for the SNAP alignment workloads (ctypes wrapper over synth.c).

This module makes inputs only; it holds none of the alignment method's arithmetic,
so the oracle and the CUDA path both consume it without sharing any logic.

Workload recipes (genome size, repeat fraction, read count and length mix, error
model, and the five Table-1 parameters s, n, d_max, c, h_max of the paper's
"SNAP algorithm parameters" table) are in ``CONFIGS``.  The paper's own data (hg19
reads simulated with wgsim, NA12878) is not available; these synthetic inputs
stand in for it with the same read lengths and error rates.

Stream seeds: genome 0, repeat families 1, reads 2, arrivals 3, request sizes 4.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None

SEED_GENOME, SEED_REPEATS, SEED_READS, SEED_ARRIVALS, SEED_SIZES = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile synth.c into libsynth.so beside it (plain gcc, no arch-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        u64, u32, dbl, i32, vp = (ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double,
                                  ctypes.c_int, ctypes.c_void_p)
        lib.synth_genome.argtypes = [vp, u64, dbl, u64, u64, u32, u32, u32, u32, dbl, i32, vp]
        lib.synth_genome.restype = i32
        lib.synth_read_lengths.argtypes = [vp, u64, i32, u32, u32, u32, dbl, u64]
        lib.synth_read_lengths.restype = i32
        lib.synth_arrivals.argtypes = [vp, vp, u64, dbl, u32, u32, u64, u64]
        lib.synth_arrivals.restype = i32
        lib.synth_reads.argtypes = [vp, u64, vp, u64, u64, dbl, dbl, u32, u32, u64, vp, vp, i32,
                                    vp, vp, vp, i32]
        lib.synth_reads.restype = i32
        lib.synth_rng_first.argtypes = [u64, vp, u64]
        lib.synth_rng_first.restype = u64
        _lib = lib
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _threads(threads: Optional[int]) -> int:
    return max(1, min(64, threads if threads else (os.cpu_count() or 1)))


def rng_first(seed: int, n: int) -> np.ndarray:
    """First n outputs of xoshiro256** seeded through splitmix64(seed)."""
    out = np.zeros(n, dtype=np.uint64)
    _load().synth_rng_first(seed, _ptr(out), n)
    return out


def genome(G: int, repeat_frac: float = 0.0, seed_genome: int = SEED_GENOME,
           seed_repeats: int = SEED_REPEATS, unit=(300, 6000), copies=(2, 50),
           divergence: float = 0.02, threads: Optional[int] = None):
    """Uniform ACGT genome plus repeat families; returns (uint8 ASCII array, covered bases)."""
    out = np.empty(G, dtype=np.uint8)
    cov = ctypes.c_uint64(0)
    rc = _load().synth_genome(_ptr(out), G, repeat_frac, seed_genome, seed_repeats, unit[0],
                              unit[1], copies[0], copies[1], divergence, _threads(threads),
                              ctypes.byref(cov))
    if rc != 0:
        raise RuntimeError(f"synth_genome failed ({rc})")
    return out, int(cov.value)


def read_lengths(n: int, mode: int, m_fixed: int = 100, lo: int = 100, hi: int = 1000,
                 frac_fixed: float = 0.0, seed: int = SEED_READS) -> np.ndarray:
    lens = np.empty(n, dtype=np.uint32)
    rc = _load().synth_read_lengths(_ptr(lens), n, mode, m_fixed, lo, hi, frac_fixed,
                                    seed ^ 0x4C454E53)
    if rc != 0:
        raise RuntimeError("synth_read_lengths failed")
    return lens


@dataclass
class Reads:
    bases: np.ndarray      # uint8 ASCII, concatenated
    offsets: np.ndarray    # uint64 [n+1]
    origin: np.ndarray     # int64 [n] true start on the forward strand
    strand: np.ndarray     # uint8 [n] 1 = read is the reverse complement
    edits: np.ndarray      # uint32 [n] number of simulated edit events

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0] - 1)

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets).astype(np.int64)

    def subset(self, idx) -> "Reads":
        idx = np.asarray(idx, dtype=np.int64)
        lens = (self.offsets[idx + 1] - self.offsets[idx]).astype(np.uint64)
        offs = np.zeros(len(idx) + 1, dtype=np.uint64)
        np.cumsum(lens, out=offs[1:])
        bases = np.empty(int(offs[-1]), dtype=np.uint8)
        for k, i in enumerate(idx):
            bases[offs[k]:offs[k + 1]] = self.bases[self.offsets[i]:self.offsets[i + 1]]
        return Reads(bases, offs, self.origin[idx], self.strand[idx], self.edits[idx])


def reads(genome_ascii: np.ndarray, lens: np.ndarray, sub_rate: float, indel_rate: float,
          indel_len=(1, 3), seed: int = SEED_READS, first_index: int = 0,
          threads: Optional[int] = None) -> Reads:
    n = int(lens.shape[0])
    lens = np.ascontiguousarray(lens, dtype=np.uint32)
    offsets = np.zeros(n + 1, dtype=np.uint64)
    if n:
        np.cumsum(lens.astype(np.uint64), out=offsets[1:])
    out = np.empty(int(offsets[-1]), dtype=np.uint8)
    origin = np.empty(n, dtype=np.int64)
    strand = np.empty(n, dtype=np.uint8)
    edits = np.empty(n, dtype=np.uint32)
    rc = _load().synth_reads(_ptr(genome_ascii), genome_ascii.shape[0], _ptr(lens), n,
                             first_index, sub_rate, indel_rate, indel_len[0], indel_len[1], seed,
                             _ptr(out), _ptr(offsets), 0, _ptr(origin), _ptr(strand), _ptr(edits),
                             _threads(threads))
    if rc != 0:
        raise RuntimeError("synth_reads failed")
    return Reads(out, offsets, origin, strand, edits)


def arrivals(n_req: int, rate: float, lo: int = 1000, hi: int = 100000):
    times = np.empty(n_req, dtype=np.float64)
    sizes = np.empty(n_req, dtype=np.uint32)
    rc = _load().synth_arrivals(_ptr(times), _ptr(sizes), n_req, rate, lo, hi, SEED_ARRIVALS,
                                SEED_SIZES)
    if rc != 0:
        raise RuntimeError("synth_arrivals failed")
    return times, sizes


# ---------------------------------------------------------------------------
# workload recipes
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class Workload:
    """One synthetic workload: genome recipe, read recipe and alignment parameters."""
    name: str
    G: int
    repeat_frac: float
    n_reads: int
    len_mode: int                 # 0 fixed, 1 log-uniform [lo,hi], 2 mix
    m_fixed: int = 100
    len_lo: int = 100
    len_hi: int = 1000
    frac_fixed: float = 0.0
    sub_rate: float = 0.01
    indel_rate: float = 0.001
    indel_len: tuple = (1, 3)
    seed_len: int = 20
    max_dist: int = 8
    max_hits: int = 300
    conf_diff: int = 2
    num_seeds: int = 0            # 0 = floor(m / s) per read
    max_dist_rule: str = "fixed"  # "fixed" | "min64_10pct" | "max8_8pct"
    extra: dict = field(default_factory=dict, compare=False, hash=False)

    def scaled(self, G: int, n_reads: int, name: Optional[str] = None) -> "Workload":
        return replace(self, G=G, n_reads=n_reads, name=name or f"{self.name}-scaled")

    def max_dist_per_read(self, lens: np.ndarray) -> Optional[np.ndarray]:
        """Per-read d_max for the uneven-length recipes; None when it is one scalar."""
        lens = np.asarray(lens, dtype=np.int64)
        if self.max_dist_rule == "fixed":
            return None
        if self.max_dist_rule == "min64_10pct":
            return np.minimum(64, lens // 10).astype(np.int32)
        if self.max_dist_rule == "max8_8pct":
            return np.maximum(8, (lens * 8 + 99) // 100).astype(np.int32)
        raise ValueError(self.max_dist_rule)

    def make_genome(self, threads: Optional[int] = None):
        return genome(self.G, self.repeat_frac, threads=threads)

    def make_lengths(self, n: Optional[int] = None) -> np.ndarray:
        return read_lengths(self.n_reads if n is None else n, self.len_mode, self.m_fixed,
                            self.len_lo, self.len_hi, self.frac_fixed)

    def make_reads(self, genome_ascii: np.ndarray, n: Optional[int] = None, first_index: int = 0,
                   lens: Optional[np.ndarray] = None, threads: Optional[int] = None) -> Reads:
        if lens is None:
            lens = self.make_lengths(n)
        return reads(genome_ascii, lens, self.sub_rate, self.indel_rate, self.indel_len,
                     first_index=first_index, threads=threads)

    def params(self) -> dict:
        return dict(max_dist=self.max_dist, max_hits=self.max_hits, conf_diff=self.conf_diff,
                    num_seeds=self.num_seeds)


CONFIGS = {
    # Plain SNAP, tiny: 1 Mbp uniform genome, 10k x 100 bp, 1% sub, 0.1% indels of 1-3.
    "C1": Workload("C1-tiny-1Mbp", G=1_000_000, repeat_frac=0.0, n_reads=10_000, len_mode=0,
                   m_fixed=100, sub_rate=0.01, indel_rate=0.001, indel_len=(1, 3), max_dist=8,
                   max_hits=300, conf_diff=2, num_seeds=5),
    # Repeat-rich mid-size: 100 Mbp, 5% repeats, 1M x 100 bp, 1% sub, 0.2% indels of 1-10.
    "C2": Workload("C2-repeat-rich-100Mbp", G=100_000_000, repeat_frac=0.05, n_reads=1_000_000,
                   len_mode=0, m_fixed=100, sub_rate=0.01, indel_rate=0.002, indel_len=(1, 10),
                   max_dist=10, max_hits=300, conf_diff=2, num_seeds=5),
    # Uneven-length batch: 400 Mbp, 5% repeats, 2M reads log-uniform [100,1000], 2% sub,
    # 0.5% indels of 1-20, d_max = min(64, floor(m/10)), n = floor(m/20).
    "C3": Workload("C3-uneven-400Mbp", G=400_000_000, repeat_frac=0.05, n_reads=2_000_000,
                   len_mode=1, len_lo=100, len_hi=1000, sub_rate=0.02, indel_rate=0.005,
                   indel_len=(1, 20), max_dist=64, max_hits=300, conf_diff=2, num_seeds=0,
                   max_dist_rule="min64_10pct"),
    # Serving loop: 3.1 Gbp, 50% repeats; 80% 100 bp, 20% log-uniform [1000,10000];
    # 5% total error, 20% of it indels (lengths 1-20); d_max = max(8, ceil(0.08 m)).
    # "5% total error" is read as 5% of bases in error: 4% substituted bases plus indel
    # events at 1%/10.5 per base (mean indel length 10.5), so about 1% of bases in indels.
    "C4": Workload("C4-serving-3.1Gbp", G=3_100_000_000, repeat_frac=0.50, n_reads=0,
                   len_mode=2, m_fixed=100, len_lo=1000, len_hi=10000, frac_fixed=0.8,
                   sub_rate=0.04, indel_rate=0.01 / 10.5, indel_len=(1, 20), max_dist=8,
                   max_hits=300,
                   conf_diff=2, num_seeds=0, max_dist_rule="max8_8pct",
                   extra=dict(req_lo=1000, req_hi=100000, n_requests=200)),
    # Human-scale throughput: same 3.1 Gbp genome, 100M x 100 bp, 1% sub, 0.1% indels of 1-5.
    "C5": Workload("C5-human-scale-3.1Gbp", G=3_100_000_000, repeat_frac=0.50,
                   n_reads=100_000_000, len_mode=0, m_fixed=100, sub_rate=0.01,
                   indel_rate=0.001, indel_len=(1, 5), max_dist=10, max_hits=300, conf_diff=2,
                   num_seeds=5),
}
