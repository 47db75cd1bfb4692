/*
 * snap.h — C-ABI of the GB300 SNAP alignment library (libsnapgpu.so).
 *
 * SNAP (Zaharia et al., "Faster and More Accurate Sequence Alignment with
 * SNAP", arXiv 1111.5572) aligns short and long DNA reads against a reference
 * genome: it cuts s-base seeds from each read, looks them up in a hash index of
 * every overlapping s-mer of the genome, votes for candidate start positions,
 * scores the most-voted candidates with an edit distance that gives up past a
 * limit, and reports the best hit as a single hit, multiple hits or not found.
 *
 * Conventions for every call:
 *   - Every function returns a SNAP_* status and never aborts the process.
 *     On failure snap_last_error() returns a message for the calling thread.
 *   - The caller owns every buffer passed in (host or device) and keeps it
 *     alive for the duration of the call (for the server: until
 *     snap_server_wait returns for that ticket).  The library owns the index
 *     and the server objects and frees them in snap_index_free /
 *     snap_server_destroy.
 *   - Bases are ASCII 'A','C','G','T' (uppercase).  Any other byte in a genome
 *     or a read makes the call fail with SNAP_E_INVAL.
 *   - Device pointers are CUDA global-memory pointers on the current device;
 *     `stream` arguments are cudaStream_t values passed as void* (NULL = the
 *     legacy default stream).
 *   - One CUDA device per process; the index lives on the device that was
 *     current when it was built, and later calls must keep that device current.
 */
#ifndef SNAP_GPU_H
#define SNAP_GPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum {
    SNAP_OK = 0,
    SNAP_E_INVAL = 1,   /* bad argument or input (non-ACGT base, size out of range) */
    SNAP_E_NOMEM = 2,   /* device or host allocation failed, or over the server budget */
    SNAP_E_CUDA = 3,    /* a CUDA runtime call or kernel failed */
    SNAP_E_TIMEOUT = 4, /* a bounded device wait gave up (status word set by a kernel) */
    SNAP_E_INTERNAL = 5 /* an internal limit or invariant failed */
};

/* Result classes of Algorithm 1 ("SNAP alignment algorithm"). */
enum { SNAP_NOT_FOUND = 0, SNAP_SINGLE_HIT = 1, SNAP_MULTIPLE_HITS = 2 };

typedef struct snap_index snap_index;   /* opaque, device-resident, library-owned */
typedef struct snap_server snap_server; /* opaque serving-loop state */

/*
 * The per-call parameters of Table "SNAP algorithm parameters" (the seed size s
 * belongs to the index):
 *   max_dist   d_max >= 0: largest edit distance reported as an alignment.
 *   max_hits   h_max in [0, 65534]: a seed with more index entries (its own
 *              occurrences plus those of its reverse complement) is skipped.
 *   conf_diff  c >= 1: a best hit is "single" only if the second best is at
 *              least c worse.
 *   num_seeds  n >= 0 seeds tried per read; 0 means floor(m / s) for a read of
 *              length m (the non-overlapping seeds).  At most m - s + 1 seeds
 *              exist; at most 2047 are used.
 *   max_dist_per_read  NULL, or one d_max per read overriding max_dist
 *              (a host pointer for snap_align / the server, a device pointer
 *              for the *_device calls).
 *   first_seeds  0 or 1: Algorithm 1, one candidate scored after each seed.
 *              k in [2, 2047]: the seeds-first variant the paper reports
 *              trying (Local Alignment, the remark after the Baeza-Yates test):
 *              the first k non-popular seeds (all of them when a read has fewer)
 *              vote before the first candidate is scored, then one candidate
 *              per seed as in Algorithm 1.
 *   collapse_duplicates  0 (default) or 1: exact-duplicate collapsing, the
 *              memoisation the paper lists as ongoing work (Ongoing Work,
 *              Approach): when the candidates a warp scores together after the
 *              Baeza-Yates test (the parallel drain of the warp-per-read kernel)
 *              include genome windows that are identical base for base on the
 *              same strand, the distance is computed once per distinct window and
 *              shared.  Results never change; snap_call_stats.ed_collapsed counts
 *              the distances it saved.  Other kernels ignore it.
 */
typedef struct {
    int32_t max_dist;
    int32_t max_hits;
    int32_t conf_diff;
    int32_t num_seeds;
    const int32_t* max_dist_per_read;
    int32_t first_seeds;
    int32_t collapse_duplicates;
} snap_params;

/*
 * One result per read, 16 bytes.  location is the 0-based genome position p
 * where the read (strand 0) or its reverse complement (strand 1) starts;
 * edit_distance is the distance found there.  Not found, and multiple hits
 * whose best distance exceeds d_max, report location = -1, strand = 0,
 * edit_distance = -1.
 */
typedef struct {
    int64_t location;
    int32_t edit_distance;
    uint8_t strand;
    uint8_t cls;
    uint8_t pad[2];
} snap_result;

typedef struct {
    uint64_t genome_len;
    int32_t seed_len;
    int32_t stride;         /* indexed windows start at multiples of this (1: every one) */
    uint64_t table_slots;     /* open-addressing slots (16 bytes each, 4 per bucket) */
    uint64_t distinct_seeds;  /* occupied slots: distinct canonical s-mers */
    uint64_t list_entries;    /* positions stored out of line (keys seen 2..65534 times) */
    uint64_t device_bytes;    /* device memory held by the index */
    double build_seconds;
} snap_index_info;

/*
 * Build the seed index of the "Hash Index" subsection: every overlapping s-mer
 * of genome_ascii[0..genome_len) (a window slid one base at a time), looked up
 * in both orientations as item 2 after Algorithm 1 asks.  The genome is copied
 * to the device, packed 2 bits per base, and kept resident with the index.
 *   genome_ascii  host pointer, genome_len bytes of A/C/G/T.
 *   genome_len    seed_len <= genome_len < 2^32 - 2^16.
 *   seed_len      s in [8, 32].
 *   out           receives the new index (NULL on failure).
 * Errors: SNAP_E_INVAL (bad base, bad sizes), SNAP_E_NOMEM, SNAP_E_CUDA.
 */
int snap_index_build(const uint8_t* genome_ascii, uint64_t genome_len, int seed_len,
                     snap_index** out);

/*
 * The same with a stride-k index (Hash Index, the Overlapping Seeds footnote:
 * sliding the window k bases at a time gives a k-times smaller index at the cost
 * of more lookups): only windows starting at multiples of `stride` are indexed,
 * and every align call on this index looks each seed up at its offset and the
 * stride - 1 offsets after it (those that fit in the read), so that an
 * error-free seed meets one indexed window whatever the alignment.  A seed votes
 * with its non-popular probes, is skipped when all are popular, and counts
 * toward Algorithm 1's "non-overlapping seeds tested" only when none of its
 * probes was popular.  stride 1 is snap_index_build.
 *   stride   k in [1, 16]; a read may use at most 2047 seeds whatever k is.
 * Errors: as snap_index_build, and SNAP_E_INVAL for a stride outside [1, 16].
 */
int snap_index_build_stride(const uint8_t* genome_ascii, uint64_t genome_len, int seed_len,
                            int stride, snap_index** out);

/* Free an index and its device memory.  NULL is accepted. */
int snap_index_free(snap_index* index);

/* Sizes of a built index. */
int snap_index_info_get(const snap_index* index, snap_index_info* out);

/*
 * Align n_reads reads with Algorithm 1 (batched form: a thread-per-read kernel
 * for short reads, then one persistent kernel per read-length class with a warp
 * or, for classes of few long reads, a block per read, the launch sequence
 * replayed from a cached CUDA graph).  Host buffers:
 *   reads_ascii   the reads back to back; read r is
 *                 reads_ascii[read_offsets[r] .. read_offsets[r+1]).
 *   read_offsets  n_reads + 1 non-decreasing entries.
 *   params        see snap_params (max_dist_per_read is a host pointer here).
 *   out           n_reads results.
 * A read shorter than the seed length is SNAP_NOT_FOUND.  Reads may be up to
 * 65535 bases long.  Errors: SNAP_E_INVAL, SNAP_E_NOMEM, SNAP_E_CUDA,
 * SNAP_E_TIMEOUT.
 */
int snap_align(const snap_index* index, const uint8_t* reads_ascii, const uint64_t* read_offsets,
               uint64_t n_reads, const snap_params* params, snap_result* out);

/* The same on device buffers, ordered on `stream`; returns once the results
 * are in d_out (the call synchronises the stream).  params->max_dist_per_read,
 * when set, is a device pointer. */
int snap_align_device(const snap_index* index, const uint8_t* d_reads, const uint64_t* d_offsets,
                      uint64_t n_reads, const snap_params* params, snap_result* d_out,
                      void* stream);

/*
 * The plain form of the same computation: one kernel launch per stage (seed
 * probe, candidate gather and dedup, edit distance of every candidate at
 * d_max + c - 1, replay of Algorithm 1's decisions), no persistent queue, no
 * graph.  Results are identical to snap_align_device's; it exists as the
 * comparison form.  Same arguments and errors.
 */
int snap_align_plain_device(const snap_index* index, const uint8_t* d_reads,
                            const uint64_t* d_offsets, uint64_t n_reads,
                            const snap_params* params, snap_result* d_out, void* stream);

/*
 * snap_align_device without any device memory allocation.  The paper has no
 * counterpart: this exists for callers that cannot let the library call
 * cudaMalloc or cudaFree, for example code running under a framework that has
 * already reserved the device memory for its own pool, a serving thread that
 * must not stall the device (cudaMalloc/cudaFree can synchronize it), or a
 * process that routes every device allocation through its own allocator.
 *
 * All scratch (batch statistics, status word, queue heads, packed reads, a list
 * of deferred reads, candidate tables that do not fit in shared memory) lives in
 * one fixed 64 MiB array that every GPU loading the library holds until the
 * process exits, whether or not this entry point is ever called.  A call runs two
 * launches: the first fills every SM and aligns each read whose candidate table
 * fits in shared memory; a read whose candidates outgrow it is listed and aligned
 * by the second launch, one table per warp in the array.  The results are those
 * of snap_align_device.
 *
 * Errors: those of snap_align_device, and SNAP_E_INVAL, before any read is
 * aligned, for
 *   - more than 201,326,432 read bases in the call (the reads are packed 4 per
 *     byte into 48 MiB): split the batch;
 *   - a seeds x max_hits bound above 262,144 for some read (one warp's table
 *     must fit in the array's 14 MiB of tables), e.g. reads longer than about
 *     17 kb at max_hits 300 with num_seeds = 0;
 * and SNAP_E_INVAL after the first launch when more than 524,288 reads of the
 * call need a table larger than shared memory (split the batch).  The caller
 * still passes (and owns) the reads, offsets and results, as for
 * snap_align_device.
 *
 * The first call on a device looks up the array's device address and caches
 * it; make that first call before any stream capture on that device.  Every
 * call synchronizes `stream` (it reads the batch statistics and the count of
 * deferred reads back) and returns once the results are in d_out.  Every call
 * reuses the same array, so calls whose GPU work overlaps (other streams, other
 * threads) race with each other: keep them ordered.
 */
int snap_align_device_noalloc(const snap_index* index, const uint8_t* d_reads,
                              const uint64_t* d_offsets, uint64_t n_reads,
                              const snap_params* params, snap_result* d_out, void* stream);

/* Host-buffer variant of the plain form. */
int snap_align_plain(const snap_index* index, const uint8_t* reads_ascii,
                     const uint64_t* read_offsets, uint64_t n_reads, const snap_params* params,
                     snap_result* out);

/*
 * Serving loop (continuous batching).  A server owns a worker thread, a set of
 * CUDA streams and a device-memory budget.  snap_server_submit enqueues a
 * request (host buffers, kept alive by the caller until snap_server_wait
 * returns for its ticket); the worker admits queued requests in arrival order
 * whenever a stream slot is free and the request's device footprint fits in
 * what is left of mem_budget_bytes, so requests that arrive while others run
 * overlap on the device.  A request larger than the whole budget fails with
 * SNAP_E_NOMEM at wait.  Results do not depend on what else is in flight.
 *   mem_budget_bytes  device bytes the server may hold for request data.
 *   max_inflight      concurrent requests on the device (1..64).
 */
int snap_server_create(const snap_index* index, uint64_t mem_budget_bytes, int max_inflight,
                       snap_server** out);
int snap_server_submit(snap_server* server, const uint8_t* reads_ascii,
                       const uint64_t* read_offsets, uint64_t n_reads, const snap_params* params,
                       uint64_t* ticket);
/* Block until request `ticket` is done; copy its results to out (n_reads of
 * them) and its latency (submit to completion, seconds) to *latency_s. */
int snap_server_wait(snap_server* server, uint64_t ticket, snap_result* out, double* latency_s);
/* Wait for every request, stop the worker and free the server.  NULL is accepted. */
int snap_server_destroy(snap_server* server);

/*
 * Measurements of the last successful align call on an index (any form):
 * device time per stage from CUDA events recorded on the call's stream, the
 * number of library kernels it launched, and traffic counters kept by the
 * kernels (index probes read 64-byte buckets of four 16-byte slots and
 * slot_reads counts the slots read; out-of-line list entries are 4 bytes; a
 * scored candidate stages its genome window).
 */
typedef struct {
    uint64_t kernel_launches;
    double stats_ms;   /* batch statistics and validation */
    double pack_ms;    /* 2-bit packing of the reads */
    double align_ms;   /* everything after packing: the main kernel(s) */
    double total_ms;
    uint64_t reads;
    uint64_t read_bases;
    uint64_t seeds;         /* seeds looked up */
    uint64_t slot_reads;    /* index slots read by the probes */
    uint64_t list_entries;  /* out-of-line positions read */
    uint64_t ed_calls;      /* edit distances computed */
    uint64_t ed_over;       /* of which over the limit */
    uint64_t window_bytes;  /* packed genome bytes staged for edit distances */
    int32_t light_threads;    /* batched form: threads per block of the thread-per-read kernel */
    int32_t warps_per_block;  /* batched form: warps per block of the warp-per-read kernel */
    int32_t table_slots;      /* batched form: shared candidate slots per warp */
    int32_t graph_replay;     /* 1 when the launch sequence ran as a CUDA graph */
    int32_t team_classes;     /* read-length classes aligned one read per block: team
                                 mode (all warps of the block on each edit distance) or
                                 wave mode (each warp on its own candidate) */
    uint64_t ed_filtered;     /* edit distances (counted in ed_calls and ed_over) proven
                                 over the limit by the q-gram bound without the rounds */
    double probe_ms;          /* plain form: the seed-probe stage kernel alone (its
                                 traffic is seeds x (8 + 16) bytes + 16 per slot read);
                                 0 for the batched form, where probes are fused */
    double distance_ms;       /* plain form: the edit-distance stage kernel alone */
    double host_plan_ms;      /* host time from the batch statistics reaching the host to
                                 the last align launch being enqueued (planning, graph
                                 update); the device idles for whatever part of it
                                 outlasts the read-packing kernel */
    /* batched form: the thread-per-read kernel alone (its share of the counters above,
       and its device time: the device clock from its first block's start to its last
       block's end) */
    double light_ms;
    uint64_t reads_light;         /* reads it finished (the rest went to the warp kernels) */
    uint64_t light_seeds;
    uint64_t light_slot_reads;
    uint64_t light_list_entries;
    uint64_t light_ed_calls;
    uint64_t light_window_bytes;
    uint64_t ed_collapsed;        /* distances taken from an identical window on the same
                                     strand (collapse_duplicates); counted in ed_calls */
    int32_t wave_classes;         /* of team_classes, those aligned in wave mode */
    int32_t wave_warps;           /* warps (candidates per wave) of the last such class */
} snap_call_stats;

int snap_last_call_stats(const snap_index* index, snap_call_stats* out);

/*
 * Options of the batched form on one index (both on by default):
 *   autotune     on the first batch of a new shape (read lengths, limits, seed
 *                count, batch size within a factor of two), time a few launch
 *                shapes (threads per block of the thread-per-read kernel, warps per
 *                block and shared candidate slots of the warp-per-read kernel) on
 *                that batch and keep the fastest for later batches of that shape.
 *                Results never depend on the shape.
 *   cuda_graphs  capture the per-batch launch sequence and replay it as one CUDA
 *                graph, updated in place between calls (only on a stream other
 *                than the legacy or per-thread default stream).
 *   team         how a read-length class whose limits exceed 31 is aligned:
 *                -1 (default) picks per batch, team mode when the class has fewer
 *                than max(8, longest read / 12) reads per SM, else one warp per
 *                read; 0 always one warp per read; 1 always team mode (one read
 *                per block of 8 warps, all of them on each edit distance); 2
 *                always wave mode (one read per block; each warp computes one of
 *                the read's next picks in Algorithm 1's order, at a bound on the
 *                limits to come, and the block's first warp replays them in
 *                order); it falls back to team mode when the index has a
 *                stride or first_seeds > 1.  Results never depend on it.
 * Passing autotune = 0 also forgets tuned shapes.  Returns SNAP_E_INVAL for a
 * NULL index or team outside -1..2.
 */
int snap_index_configure(snap_index* index, int autotune, int cuda_graphs, int team);

/* Measurement helper; Algorithm 1 has no counterpart.  Every index probe,
 * position-list read and genome-window fetch of the aligner reads a few dozen
 * bytes at an unpredictable address, so the streaming-copy bandwidth of HBM
 * overstates what that traffic can reach.  This measures the random-gather
 * ceiling on the current device: about n_reads independent reads of one
 * chunk_bytes-aligned chunk (16, 32 or 64 bytes) at pseudo-random chunk indices of a
 * device buffer of buffer_bytes (>= 64 MiB; make it far larger than L2),
 * 2048 threads per SM, chunk_bytes / 16 threads on each chunk and 4 chunks in
 * flight per thread; best of three timed runs
 * after one warm-up.  Writes the delivered chunk bytes per second / 1e9 to
 * *gbs_out.  Allocates and frees the buffer itself; SNAP_E_NOMEM when it does
 * not fit, SNAP_E_INVAL for other sizes. */
int snap_measure_gather(uint64_t buffer_bytes, uint32_t chunk_bytes, uint64_t n_reads,
                        double* gbs_out);

/* The same measurement with its launch shape as arguments, to find the ceiling
 * rather than one point under it: chunk_bytes 16, 32, 64 or 128; ilp = chunks in
 * flight per thread (1, 2, 4, 8 or 16); threads_per_sm a multiple of 256 in
 * [256, 2048].  snap_measure_gather is ilp 4 at 2048 threads per SM.  Errors as
 * snap_measure_gather (SNAP_E_INVAL for other shapes). */
int snap_measure_gather_config(uint64_t buffer_bytes, uint32_t chunk_bytes, uint64_t n_reads,
                               int ilp, int threads_per_sm, double* gbs_out);

/* Message for the last failed call on this thread ("" if none). */
const char* snap_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SNAP_GPU_H */
