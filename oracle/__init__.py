"""CPU oracle for the SNAP alignment path (ctypes wrapper over snap_oracle.cpp).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and bench.py's
cpu_baseline and reference legs may import this package.  The CUDA product path in
``paper_1111_5572_gb300`` never imports, links or runs it, and the two share no code.

The oracle is a plain, slow, single-read-at-a-time restatement of the paper's
method: the overlapping-seed hash index (Methods, "Hash Index"), the seed order
(item 3 after Algorithm 1), the bounded edit distance (Methods, "Local Alignment")
and Algorithm 1 itself with the 32-base bucket merge.  The readings it takes where
the paper is silent are listed at the top of snap_oracle.cpp.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "snap_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

NOT_FOUND, SINGLE_HIT, MULTIPLE_HITS = 0, 1, 2

RESULT_DTYPE = np.dtype([("location", "<i8"), ("edit_distance", "<i4"), ("strand", "u1"),
                         ("cls", "u1"), ("pad", "u1", (2,))])
assert RESULT_DTYPE.itemsize == 16


class _Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "reads", "seeds_looked_up", "seeds_popular", "ed_calls", "ed_over",
        "ed_calls_after_first", "ed_over_after_first", "reads_with_hit",
        "first_scored_is_best", "candidates", "n_not_found", "n_single", "n_multiple")]


def build(force: bool = False) -> str:
    """Compile snap_oracle.cpp into liboracle.so beside it (plain g++)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp, u64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
        lib.or_index_build.argtypes = [vp, u64, i32, i32, vp, u64, ctypes.POINTER(ctypes.c_int)]
        lib.or_index_build.restype = vp
        lib.or_index_free.argtypes = [vp]
        lib.or_index_free.restype = None
        lib.or_index_entries.argtypes = [vp]
        lib.or_index_entries.restype = u64
        lib.or_index_occurrences.argtypes = [vp, vp, vp, u64]
        lib.or_index_occurrences.restype = u64
        lib.or_seed_offsets.argtypes = [i32, i32, i32, vp, vp, i32]
        lib.or_seed_offsets.restype = i32
        lib.or_ed_lv.argtypes = [vp, i32, vp, i32, i32]
        lib.or_ed_lv.restype = i32
        lib.or_ed_dp.argtypes = [vp, i32, vp, i32]
        lib.or_ed_dp.restype = i32
        lib.or_ed_pairs.argtypes = [vp, vp, vp, vp, vp, u64, vp, vp]
        lib.or_ed_pairs.restype = None
        lib.or_read_seed_kmers.argtypes = [vp, vp, u64, i32, i32, i32, vp, u64]
        lib.or_read_seed_kmers.restype = u64
        lib.or_align.argtypes = [vp, vp, vp, u64, i32, i32, i32, i32, i32, vp, i32, i32, vp,
                                 ctypes.POINTER(_Stats)]
        lib.or_align.restype = i32
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _bytes(x) -> np.ndarray:
    if isinstance(x, (bytes, bytearray)):
        return np.frombuffer(bytes(x), dtype=np.uint8).copy()
    if isinstance(x, str):
        return np.frombuffer(x.encode(), dtype=np.uint8).copy()
    return np.ascontiguousarray(x, dtype=np.uint8)


def ed_lv(x, t, L: int) -> int:
    """Bounded distance of X against a free-ended prefix of T; -1 when over L."""
    xa, ta = _bytes(x), _bytes(t)
    return int(_load().or_ed_lv(_p(xa), len(xa), _p(ta), len(ta), L))


def ed_dp(x, t) -> int:
    """min over j of Lev(X, T[0..j)) by the full O(|X||T|) table."""
    xa, ta = _bytes(x), _bytes(t)
    return int(_load().or_ed_dp(_p(xa), len(xa), _p(ta), len(ta)))


def _concat(strs):
    arrs = [_bytes(x) for x in strs]
    off = np.zeros(len(arrs) + 1, dtype=np.uint64)
    if arrs:
        np.cumsum([a.shape[0] for a in arrs], out=off[1:])
    buf = np.concatenate(arrs) if arrs and off[-1] > 0 else np.zeros(1, dtype=np.uint8)
    return np.ascontiguousarray(buf, dtype=np.uint8), off


def ed_pairs(xs, ts, Ls, with_dp: bool = True):
    """Batch form of ed_lv / ed_dp over lists of strings; returns (lv, dp) int32 arrays."""
    n = len(xs)
    xb, xo = _concat(xs)
    tb, to = _concat(ts)
    L = np.ascontiguousarray(Ls, dtype=np.int32)
    lv = np.zeros(n, dtype=np.int32)
    dp = np.zeros(n, dtype=np.int32) if with_dp else None
    _load().or_ed_pairs(_p(xb), _p(xo), _p(tb), _p(to), _p(L), n, _p(lv), _p(dp))
    return lv, dp


def seed_offsets(m: int, s: int, n: int):
    cap = max(1, m)
    offs = np.zeros(cap, dtype=np.int32)
    p0 = np.zeros(cap, dtype=np.uint8)
    k = _load().or_seed_offsets(m, s, n, _p(offs), _p(p0), cap)
    return offs[:k].tolist(), p0[:k].astype(bool).tolist()


def read_seed_kmers(bases: np.ndarray, offsets: np.ndarray, s: int, n_seeds: int,
                    stride: int = 1) -> np.ndarray:
    lib = _load()
    n = int(offsets.shape[0] - 1)
    need = lib.or_read_seed_kmers(_p(bases), _p(offsets), n, s, n_seeds, stride, None, 0)
    out = np.zeros(max(1, need), dtype=np.uint64)
    lib.or_read_seed_kmers(_p(bases), _p(offsets), n, s, n_seeds, stride, _p(out), need)
    return np.unique(out[:need])


@dataclass
class Stats:
    reads: int
    seeds_looked_up: int
    seeds_popular: int
    ed_calls: int
    ed_over: int
    ed_calls_after_first: int
    ed_over_after_first: int
    reads_with_hit: int
    first_scored_is_best: int
    candidates: int
    n_not_found: int
    n_single: int
    n_multiple: int


class Index:
    """Sorted-array index of every overlapping s-mer (optionally restricted to a key set)."""

    def __init__(self, genome_ascii: np.ndarray, seed_len: int,
                 kmer_filter: Optional[np.ndarray] = None, stride: int = 1):
        lib = _load()
        self._genome = np.ascontiguousarray(genome_ascii, dtype=np.uint8)
        err = ctypes.c_int(0)
        filt = None if kmer_filter is None else np.ascontiguousarray(kmer_filter, dtype=np.uint64)
        t0 = time.perf_counter()
        h = lib.or_index_build(_p(self._genome), self._genome.shape[0], seed_len, int(stride),
                               _p(filt), 0 if filt is None else filt.shape[0], ctypes.byref(err))
        self.build_seconds = time.perf_counter() - t0
        if not h:
            raise ValueError(f"oracle index build failed (code {err.value})")
        self._h = h
        self.seed_len = seed_len
        self.stride = int(stride)
        self.G = int(self._genome.shape[0])

    @property
    def entries(self) -> int:
        return int(_load().or_index_entries(self._h))

    def occurrences(self, smer) -> list:
        a = _bytes(smer)
        cap = 1 << 16
        out = np.zeros(cap, dtype=np.uint32)
        n = int(_load().or_index_occurrences(self._h, _p(a), _p(out), cap))
        return out[:min(n, cap)].tolist()

    def align(self, bases: np.ndarray, offsets: np.ndarray, max_dist: int = 8,
              max_hits: int = 300, conf_diff: int = 2, num_seeds: int = 0,
              max_dist_per_read: Optional[np.ndarray] = None, mode: int = 0,
              threads: int = 1, first_seeds: int = 0):
        """Align reads; returns (results structured array, Stats).  first_seeds > 1 runs
        the seeds-first variant (that many non-popular seeds vote before the first
        candidate is scored)."""
        bases = np.ascontiguousarray(bases, dtype=np.uint8)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        n = int(offsets.shape[0] - 1)
        out = np.zeros(n, dtype=RESULT_DTYPE)
        dpr = None if max_dist_per_read is None else np.ascontiguousarray(max_dist_per_read,
                                                                          dtype=np.int32)
        st = _Stats()
        rc = _load().or_align(self._h, _p(bases), _p(offsets), n, max_dist, max_hits, conf_diff,
                              num_seeds, first_seeds, _p(dpr), mode, threads, _p(out),
                              ctypes.byref(st))
        if rc != 0:
            raise ValueError("oracle align: invalid input (non-ACGT base)")
        return out, Stats(**{f: int(getattr(st, f)) for f, _ in _Stats._fields_})

    def close(self):
        if getattr(self, "_h", None):
            _load().or_index_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
