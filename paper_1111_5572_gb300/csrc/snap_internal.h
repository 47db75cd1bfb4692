// snap_internal.h — library-private definitions shared by the host and device
// code of libsnapgpu.so.  Nothing here is part of the C-ABI (include/snap.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "snap.h"

namespace snapgpu {

// ---- sizes and limits ------------------------------------------------------
constexpr unsigned long long kEmptyKey = ~0ull;  // never a canonical s-mer (see snap_index.cu)
constexpr uint32_t kListMax = 65534;             // longest stored position list; max h_max
constexpr int kMaxSeeds = 2047;                  // seeds per read (11-bit vote counter)
constexpr int kMaxStride = 16;                   // stride-k index: largest k
constexpr int kMaxReadLen = 65535;
constexpr int kReadPadBases = 32;                // packed read stream starts 32 bases in
constexpr uint32_t kMaxTableSlots = 1u << 20;    // per-read candidate table (20-bit slot id)

// Status word bits written by kernels (host maps them to SNAP_E_*).
enum : int {
    kStBadBase = 1 << 0,
    kStBadOffsets = 1 << 1,
    kStReadTooLong = 1 << 2,
    kStTooManySeeds = 1 << 3,
    kStTableFull = 1 << 4,
    kStProbeRunaway = 1 << 5,
    kStBadDmax = 1 << 6,
    kStInternal = 1 << 7,
    kStTimeout = 1 << 8,
};

// One open-addressing slot of the seed index, 16 bytes.  key = canonical
// s-mer (min of the s-mer and its reverse complement, 2 bits per base, first
// base in the low bits).  A = positions where the genome reads `key`,
// B = positions where it reads revcomp(key).  When nA + nB == 1 the single
// position is stored inline in `field`; when 2 <= nA + nB <= kListMax,
// positions[field .. field+nA) = A and positions[field+nA .. +nB) = B.
// Counts saturate at 65535.  During the build the same 16 bytes hold
// {key, countA(u32), countB(u32)}.
struct __align__(16) IndexSlot {
    unsigned long long key;
    uint32_t field;
    uint16_t nA;
    uint16_t nB;
};
static_assert(sizeof(IndexSlot) == 16, "slot is one 16-byte vector");

// Per-seed record of the read being aligned (16 bytes).  The two lists are the
// forward occurrences of the seed S (strand-0 votes) and of revcomp(S)
// (strand-1 votes), each inline (one position in *_ref) or out of line.
struct __align__(16) SeedRec {
    uint32_t fwd_ref;
    uint32_t rc_ref;
    uint16_t fwd_n;
    uint16_t rc_n;
    uint16_t offset;
    uint8_t flags;  // kSeed* bits
    uint8_t pad;
};
static_assert(sizeof(SeedRec) == 16, "seed record is 16 bytes");
enum : uint8_t { kSeedPopular = 1, kSeedPass0 = 2, kSeedFwdInline = 4, kSeedRcInline = 8,
                 kSeedValid = 16,
                 kSeedPick = 32,     // pick and score after this probe's votes (its seed's last
                                     // non-popular probe)
                 kSeedCountT = 64 };  // this probe's seed counts toward t

// Candidate table slot of one read (16 bytes): key = 2p + strand.
struct __align__(16) CandSlot {
    unsigned long long key;
    uint32_t votes;
    int32_t state;  // kUnscored, kOver, or the distance found (>= 0)
};
constexpr int32_t kUnscored = -2;
constexpr int32_t kOver = -1;

struct HitRec {
    unsigned long long key;
    int32_t d;
    int32_t pad;
};

// Traffic counters accumulated by the align kernels (one atomicAdd per warp).
struct DevCounters {
    unsigned long long seeds, slot_reads, list_entries, ed_calls, ed_over, window_words,
        ed_filtered, reads_done, ed_collapsed;
};

// Statistics of a read batch, computed on the device before the main launch.
struct BatchStats {
    unsigned long long total_bases;
    unsigned int max_len;
    int max_L0;        // max over reads of d_max + c - 1
    int max_seeds;     // max over reads of n
    int status;
    unsigned long long max_hits_bound;  // max over reads of n * h_max (capped)
    DevCounters ctr;        // every align kernel of the call (both forms)
    DevCounters ctr_light;  // the thread-per-read kernel alone (also in ctr)
    // device clock (ns) of the thread-per-read kernel: the latest block end, and the
    // complement of the earliest block start (atomicMax of ~start is a min of start)
    unsigned long long light_end_ns, light_start_ns_neg;
    unsigned long long n_light;  // reads short enough for the thread-per-read bucket
    // per read-length class (see kClassBounds): reads and the maxima that size a launch
    unsigned long long cls_n[4];
    unsigned int cls_max_len[4];
    int cls_max_L0[4];
    int cls_max_seeds[4];
    unsigned long long cls_max_hits[4];
};
// read-length classes of the warp-per-read kernel: m <= 256, <= 1024, <= 4096, longer
constexpr int kClasses = 4;
__host__ __device__ inline int length_class(uint64_t m) {
    return (m > 256) + (m > 1024) + (m > 4096);
}

}  // namespace snapgpu

// ---- library-owned objects --------------------------------------------------
namespace snapgpu {
struct Engine;  // per-index align workspaces and cached graphs (snap_align.cu)
}

struct snap_index {
    int device = 0;
    uint64_t G = 0;
    int s = 0;
    int stride = 1;                    // indexed windows start at multiples of this
    uint32_t* genome_words = nullptr;  // 2-bit packed genome, padded
    uint64_t genome_words_n = 0;
    snapgpu::IndexSlot* slots = nullptr;
    uint64_t T = 0;
    uint32_t* positions = nullptr;
    uint64_t n_positions = 0;
    uint64_t distinct = 0;
    uint64_t device_bytes = 0;
    double build_seconds = 0;
    snapgpu::Engine* engine = nullptr;
};

namespace snapgpu {

// thread-local last error
void set_error(const char* fmt, ...);
void clear_error();
int cuda_fail(cudaError_t e, const char* what);
int raise_smem_limit(const void* func, size_t bytes);  // never lowers it

// Held while a stream is being captured into a CUDA graph and around every
// device or pinned allocation and free.  cudaFree / cudaFreeHost wait for the
// whole device, which would be an implicit synchronisation with a stream that
// another thread (a serving slot) is capturing and would invalidate its graph.
std::recursive_mutex& capture_alloc_mutex();

#define SNAP_CUDA(call, what)                                  \
    do {                                                       \
        cudaError_t _e = (call);                               \
        if (_e != cudaSuccess) return ::snapgpu::cuda_fail(_e, what); \
    } while (0)

// host helpers implemented in snap_align.cu
int validate_params(const snap_index* idx, const snap_params* p);
int status_to_code(int st, const char* where);
void shift_list(int s, uint8_t* out, int* n_out);

// grow-only device buffer
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    int ensure(size_t need, const char* what);
    void release();
};

struct PinnedBuf {
    void* p = nullptr;
    size_t bytes = 0;
    int ensure(size_t need, const char* what);
    void release();
};

// Align one batch on `stream` with the batched (persistent) or plain form.
// Device pointers; blocks until done.
int align_batch_device(const snap_index* idx, Engine* eng, const uint8_t* d_reads,
                       const uint64_t* d_offsets, uint64_t n_reads, const snap_params* p,
                       snap_result* d_out, cudaStream_t stream, bool plain);

Engine* engine_create();
void engine_destroy(Engine* e);
size_t engine_bytes(const Engine* e);
void engine_release(Engine* e);  // frees the workspaces (kept: streams, events, tuning)

}  // namespace snapgpu
