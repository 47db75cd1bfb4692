"""Python binding of libsnapgpu.so, the GB300 SNAP alignment library (include/snap.h).

Argument marshalling only: every step of the alignment runs in the library's CUDA
kernels.  PyTorch is used for device memory and streams in the *_device calls; host
calls take numpy arrays.  If the library has not been built the calls raise
``RuntimeError`` (there is no fallback of any kind).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsnapgpu.so")

SNAP_OK, SNAP_E_INVAL, SNAP_E_NOMEM, SNAP_E_CUDA, SNAP_E_TIMEOUT, SNAP_E_INTERNAL = range(6)
NOT_FOUND, SINGLE_HIT, MULTIPLE_HITS = 0, 1, 2

RESULT_DTYPE = np.dtype([("location", "<i8"), ("edit_distance", "<i4"), ("strand", "u1"),
                         ("cls", "u1"), ("pad", "u1", (2,))])
assert RESULT_DTYPE.itemsize == 16

# every symbol include/snap.h declares
EXPORTS = ("snap_index_build", "snap_index_build_stride", "snap_index_free", "snap_index_info_get", "snap_align",
           "snap_align_device", "snap_align_plain_device", "snap_align_plain",
           "snap_server_create", "snap_server_submit", "snap_server_wait", "snap_server_destroy",
           "snap_last_call_stats", "snap_align_device_noalloc", "snap_index_configure",
           "snap_measure_gather", "snap_measure_gather_config",
           "snap_last_error")


class SnapError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"SNAP error {code}: {msg}")
        self.code = code


class snap_params(ctypes.Structure):
    _fields_ = [("max_dist", ctypes.c_int32), ("max_hits", ctypes.c_int32),
                ("conf_diff", ctypes.c_int32), ("num_seeds", ctypes.c_int32),
                ("max_dist_per_read", ctypes.c_void_p), ("first_seeds", ctypes.c_int32),
                ("collapse_duplicates", ctypes.c_int32)]


class snap_index_info(ctypes.Structure):
    _fields_ = [("genome_len", ctypes.c_uint64), ("seed_len", ctypes.c_int32),
                ("stride", ctypes.c_int32), ("table_slots", ctypes.c_uint64),
                ("distinct_seeds", ctypes.c_uint64), ("list_entries", ctypes.c_uint64),
                ("device_bytes", ctypes.c_uint64), ("build_seconds", ctypes.c_double)]


class snap_call_stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_uint64), ("stats_ms", ctypes.c_double),
                ("pack_ms", ctypes.c_double), ("align_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double), ("reads", ctypes.c_uint64),
                ("read_bases", ctypes.c_uint64), ("seeds", ctypes.c_uint64),
                ("slot_reads", ctypes.c_uint64), ("list_entries", ctypes.c_uint64),
                ("ed_calls", ctypes.c_uint64), ("ed_over", ctypes.c_uint64),
                ("window_bytes", ctypes.c_uint64), ("light_threads", ctypes.c_int32),
                ("warps_per_block", ctypes.c_int32), ("table_slots", ctypes.c_int32),
                ("graph_replay", ctypes.c_int32), ("team_classes", ctypes.c_int32),
                ("ed_filtered", ctypes.c_uint64), ("probe_ms", ctypes.c_double),
                ("distance_ms", ctypes.c_double), ("host_plan_ms", ctypes.c_double),
                ("light_ms", ctypes.c_double), ("reads_light", ctypes.c_uint64),
                ("light_seeds", ctypes.c_uint64), ("light_slot_reads", ctypes.c_uint64),
                ("light_list_entries", ctypes.c_uint64), ("light_ed_calls", ctypes.c_uint64),
                ("light_window_bytes", ctypes.c_uint64), ("ed_collapsed", ctypes.c_uint64),
                ("wave_classes", ctypes.c_int32), ("wave_warps", ctypes.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libsnapgpu.so (raises RuntimeError when it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run `python -c 'import __graft_entry__ as g; "
                           f"g.build()'` first (the CUDA library is required, there is no "
                           f"CPU fallback)")
    lib = ctypes.CDLL(path)
    vp, u64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
    P = ctypes.POINTER
    lib.snap_index_build.argtypes = [vp, u64, i32, P(vp)]
    lib.snap_index_build_stride.argtypes = [vp, u64, i32, i32, P(vp)]
    lib.snap_index_free.argtypes = [vp]
    lib.snap_index_info_get.argtypes = [vp, P(snap_index_info)]
    for name in ("snap_align", "snap_align_plain"):
        getattr(lib, name).argtypes = [vp, vp, vp, u64, P(snap_params), vp]
    for name in ("snap_align_device", "snap_align_plain_device", "snap_align_device_noalloc"):
        getattr(lib, name).argtypes = [vp, vp, vp, u64, P(snap_params), vp, vp]
    lib.snap_server_create.argtypes = [vp, u64, i32, P(vp)]
    lib.snap_server_submit.argtypes = [vp, vp, vp, u64, P(snap_params), P(u64)]
    lib.snap_server_wait.argtypes = [vp, u64, vp, P(ctypes.c_double)]
    lib.snap_server_destroy.argtypes = [vp]
    lib.snap_last_call_stats.argtypes = [vp, P(snap_call_stats)]
    lib.snap_index_configure.argtypes = [vp, i32, i32, i32]
    lib.snap_measure_gather.argtypes = [u64, ctypes.c_uint32, u64, P(ctypes.c_double)]
    lib.snap_measure_gather_config.argtypes = [u64, ctypes.c_uint32, u64, i32, i32,
                                               P(ctypes.c_double)]
    lib.snap_last_error.argtypes = []
    lib.snap_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name != "snap_last_error":
            getattr(lib, name).restype = i32
    _lib = lib
    return lib


def _check(rc: int, what: str):
    if rc != SNAP_OK:
        msg = load_library().snap_last_error().decode(errors="replace")
        raise SnapError(rc, f"{what}: {msg}")


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def make_params(max_dist: int = 8, max_hits: int = 300, conf_diff: int = 2, num_seeds: int = 0,
                max_dist_per_read_ptr: Optional[int] = None, first_seeds: int = 0,
                collapse_duplicates: int = 0) -> snap_params:
    return snap_params(int(max_dist), int(max_hits), int(conf_diff), int(num_seeds),
                       max_dist_per_read_ptr, int(first_seeds), int(collapse_duplicates))


def measure_gather(buffer_bytes: int = 8 << 30, chunk_bytes: int = 32,
                   n_reads: int = 1 << 28) -> float:
    """snap_measure_gather: GB/s delivered by independent random reads of one aligned
    chunk each (the practical ceiling of index probes and window fetches)."""
    out = ctypes.c_double()
    _check(load_library().snap_measure_gather(int(buffer_bytes), int(chunk_bytes), int(n_reads),
                                              ctypes.byref(out)), "snap_measure_gather")
    return out.value


def measure_gather_config(buffer_bytes: int = 8 << 30, chunk_bytes: int = 64,
                          n_reads: int = 1 << 28, ilp: int = 4, threads_per_sm: int = 2048) -> float:
    """snap_measure_gather_config: the same measurement at a given launch shape."""
    out = ctypes.c_double()
    _check(load_library().snap_measure_gather_config(int(buffer_bytes), int(chunk_bytes),
                                                     int(n_reads), int(ilp), int(threads_per_sm),
                                                     ctypes.byref(out)),
           "snap_measure_gather_config")
    return out.value


class Index:
    """Device-resident seed index of one genome (snap_index_build)."""

    def __init__(self, genome_ascii: np.ndarray, seed_len: int = 20, stride: int = 1):
        lib = load_library()
        g = np.ascontiguousarray(genome_ascii, dtype=np.uint8)
        h = ctypes.c_void_p()
        if stride == 1:
            _check(lib.snap_index_build(_p(g), g.shape[0], int(seed_len), ctypes.byref(h)),
                   "snap_index_build")
        else:
            _check(lib.snap_index_build_stride(_p(g), g.shape[0], int(seed_len), int(stride),
                                               ctypes.byref(h)), "snap_index_build_stride")
        self._h = h
        self.seed_len = seed_len
        self.stride = int(stride)
        self.G = int(g.shape[0])

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = snap_index_info()
        _check(load_library().snap_index_info_get(self._h, ctypes.byref(inf)), "info")
        return {f: getattr(inf, f) for f, _ in snap_index_info._fields_}

    def configure(self, autotune: bool = True, cuda_graphs: bool = True, team: int = -1):
        """snap_index_configure: autotuning of launch shapes, CUDA-graph replay and the
        block-per-read modes of long-read classes (-1 chosen per batch, 0 never,
        1 team mode, 2 wave mode)."""
        _check(load_library().snap_index_configure(self._h, int(autotune), int(cuda_graphs),
                                                   int(team)),
               "snap_index_configure")

    def last_call_stats(self) -> dict:
        """Stage timings and traffic counters of the last align call on this index."""
        cs = snap_call_stats()
        _check(load_library().snap_last_call_stats(self._h, ctypes.byref(cs)),
               "snap_last_call_stats")
        return {f: getattr(cs, f) for f, _ in snap_call_stats._fields_}

    def align(self, bases: np.ndarray, offsets: np.ndarray, max_dist: int = 8,
              max_hits: int = 300, conf_diff: int = 2, num_seeds: int = 0,
              max_dist_per_read: Optional[np.ndarray] = None, plain: bool = False,
              out: Optional[np.ndarray] = None, first_seeds: int = 0,
              collapse_duplicates: int = 0) -> np.ndarray:
        """Host buffers in, host results out (snap_align / snap_align_plain)."""
        bases = np.ascontiguousarray(bases, dtype=np.uint8)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        n = int(offsets.shape[0] - 1)
        if out is None:
            out = np.zeros(n, dtype=RESULT_DTYPE)
        dpr = None if max_dist_per_read is None else np.ascontiguousarray(max_dist_per_read,
                                                                          dtype=np.int32)
        prm = make_params(max_dist, max_hits, conf_diff, num_seeds,
                          None if dpr is None else dpr.ctypes.data, first_seeds,
                          collapse_duplicates)
        fn = load_library().snap_align_plain if plain else load_library().snap_align
        _check(fn(self._h, _p(bases), _p(offsets), n, ctypes.byref(prm), _p(out)),
               "snap_align_plain" if plain else "snap_align")
        return out

    def align_device(self, d_bases, d_offsets, d_out, max_dist: int = 8, max_hits: int = 300,
                     conf_diff: int = 2, num_seeds: int = 0, d_max_dist_per_read=None,
                     stream=None, plain: bool = False, first_seeds: int = 0,
                     collapse_duplicates: int = 0):
        """Device tensors (torch, uint8 / int64 / 16-byte rows) on `stream` (torch.cuda.Stream)."""
        n = int(d_offsets.numel() - 1)
        prm = make_params(max_dist, max_hits, conf_diff, num_seeds,
                          None if d_max_dist_per_read is None else d_max_dist_per_read.data_ptr(),
                          first_seeds, collapse_duplicates)
        st = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        fn = (load_library().snap_align_plain_device if plain
              else load_library().snap_align_device)
        _check(fn(self._h, ctypes.c_void_p(d_bases.data_ptr()),
                  ctypes.c_void_p(d_offsets.data_ptr()), n, ctypes.byref(prm),
                  ctypes.c_void_p(d_out.data_ptr()), st),
               "snap_align_plain_device" if plain else "snap_align_device")
        return d_out

    def align_device_noalloc(self, d_bases, d_offsets, d_out, max_dist: int = 8,
                             max_hits: int = 300, conf_diff: int = 2, num_seeds: int = 0,
                             d_max_dist_per_read=None, stream=None, first_seeds: int = 0,
                             collapse_duplicates: int = 0):
        """snap_align_device_noalloc: the library allocates no device memory for this call
        (for callers that must not see cudaMalloc/cudaFree); limits in include/snap.h."""
        n = int(d_offsets.numel() - 1)
        prm = make_params(max_dist, max_hits, conf_diff, num_seeds,
                          None if d_max_dist_per_read is None else d_max_dist_per_read.data_ptr(),
                          first_seeds, collapse_duplicates)
        st = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        _check(load_library().snap_align_device_noalloc(
            self._h, ctypes.c_void_p(d_bases.data_ptr()), ctypes.c_void_p(d_offsets.data_ptr()),
            n, ctypes.byref(prm), ctypes.c_void_p(d_out.data_ptr()), st),
            "snap_align_device_noalloc")
        return d_out

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.snap_index_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server over one index (snap_server_*)."""

    def __init__(self, index: Index, mem_budget_bytes: int, max_inflight: int = 4):
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.snap_server_create(index.handle, int(mem_budget_bytes), int(max_inflight),
                                      ctypes.byref(h)), "snap_server_create")
        self._h = h
        self._keep = {}

    def submit(self, bases: np.ndarray, offsets: np.ndarray, max_dist: int = 8,
               max_hits: int = 300, conf_diff: int = 2, num_seeds: int = 0,
               max_dist_per_read: Optional[np.ndarray] = None, first_seeds: int = 0,
               collapse_duplicates: int = 0) -> int:
        bases = np.ascontiguousarray(bases, dtype=np.uint8)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        dpr = None if max_dist_per_read is None else np.ascontiguousarray(max_dist_per_read,
                                                                          dtype=np.int32)
        prm = make_params(max_dist, max_hits, conf_diff, num_seeds,
                          None if dpr is None else dpr.ctypes.data, first_seeds,
                          collapse_duplicates)
        t = ctypes.c_uint64()
        _check(load_library().snap_server_submit(self._h, _p(bases), _p(offsets),
                                                 int(offsets.shape[0] - 1), ctypes.byref(prm),
                                                 ctypes.byref(t)), "snap_server_submit")
        # the caller's buffers must stay alive until wait() returns
        self._keep[int(t.value)] = (bases, offsets, dpr, prm)
        return int(t.value)

    def wait(self, ticket: int):
        bases, offsets, dpr, prm = self._keep[ticket]
        out = np.zeros(int(offsets.shape[0] - 1), dtype=RESULT_DTYPE)
        lat = ctypes.c_double()
        try:
            _check(load_library().snap_server_wait(self._h, ticket, _p(out), ctypes.byref(lat)),
                   "snap_server_wait")
        finally:
            self._keep.pop(ticket, None)
        return out, float(lat.value)

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _check(_lib.snap_server_destroy(self._h), "snap_server_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
