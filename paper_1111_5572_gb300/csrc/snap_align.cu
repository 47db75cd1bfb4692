// snap_align.cu — the batched alignment path: read packing, batch statistics
// and the persistent warp-per-read kernel that runs Algorithm 1 ("SNAP
// alignment algorithm") literally for each read it pulls from a device queue.
//
// Per read, one warp (or, in team mode, one block whose first warp does this):
//   * packs the read and its reverse complement (2 bits per base) into shared
//     memory;
//   * cuts the seeds in the order of item 3 after Algorithm 1 and probes the
//     index for all of them at once (one lane per probe: a seed has one probe,
//     or k of them on a stride-k index);
//   * walks the seeds in order: adds the votes SeedsHitting[p] of a seed with
//     at most h_max entries (lanes over list entries, a shared-memory hash
//     table keyed by (strand, p)), picks the most-voted unscored candidate
//     (warp arg-max, ties to the smaller key), computes d_limit, scores it with
//     the Landau-Vishkin edit distance (behind the q-gram bound for large
//     limits), keeps d_best / d_second over 32-base buckets (item 1 after
//     Algorithm 1), and takes the early exits; after the Baeza-Yates test the
//     remaining candidates are scored 32 at a time (the parallel drain);
//   * classifies the read (single / multiple / not found).
// Readings where the paper is silent (all shared with the oracle's statement
// of them): votes from revcomp(seed) go to strand 1 at p = l - (m - o - s);
// candidates with p < 0 are dropped; the edit distance is anchored at p with
// a free end; the "non-overlapping seeds tested" counter counts non-popular
// seeds of the first (unshifted) pass; after the Baeza-Yates test passes, all
// remaining candidates are scored in pick order and seeding stops.
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "snap_device.cuh"
#include "snap_engine.h"
#include "snap_internal.h"
#include "snap_scan.cuh"

namespace snapgpu {

constexpr int kInf = 1 << 28;
constexpr unsigned long long kKeyMask = (1ull << 33) - 1;

// ---------------------------------------------------------------------------
// batch statistics and validation
// ---------------------------------------------------------------------------
// Partial statistics of one warp (reduced across the block in shared memory
// before one set of atomics per block).
struct StatsPart {
    unsigned long long hits, light;
    unsigned long long c_n[kClasses], c_hits[kClasses];
    unsigned int len, c_len[kClasses];
    int bad, L0, nseeds, c_L0[kClasses], c_seeds[kClasses];
};

__device__ __forceinline__ void stats_merge(StatsPart& a, const StatsPart& b) {
    a.bad |= b.bad;
    a.len = max(a.len, b.len);
    a.L0 = max(a.L0, b.L0);
    a.nseeds = max(a.nseeds, b.nseeds);
    a.hits = b.hits > a.hits ? b.hits : a.hits;
    a.light += b.light;
#pragma unroll
    for (int q = 0; q < kClasses; ++q) {
        a.c_n[q] += b.c_n[q];
        a.c_len[q] = max(a.c_len[q], b.c_len[q]);
        a.c_L0[q] = max(a.c_L0[q], b.c_L0[q]);
        a.c_seeds[q] = max(a.c_seeds[q], b.c_seeds[q]);
        a.c_hits[q] = b.c_hits[q] > a.c_hits[q] ? b.c_hits[q] : a.c_hits[q];
    }
}

constexpr int kStatsThreads = 256;

// Grid of the statistics kernel: a few blocks per SM (each block merges its
// threads' partials before its atomics, so fewer blocks mean fewer atomics on
// the same few addresses).
inline unsigned stats_grid(int sms, uint64_t n) {
    uint64_t want = (n + kStatsThreads - 1) / kStatsThreads;
    const uint64_t cap = (uint64_t)sms * 4;
    return (unsigned)std::max<uint64_t>(1, std::min(want, cap));
}

__global__ void __launch_bounds__(kStatsThreads)
k_read_stats(const uint64_t* __restrict__ offsets, uint64_t n, int s, int stride, int num_seeds,
             int d_max, int c, int h_max, const int32_t* __restrict__ dmax_per_read,
             BatchStats* st) {
    StatsPart my;
    memset(&my, 0, sizeof(my));
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n;
         r += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t a = offsets[r], b = offsets[r + 1];
        if (b < a) {
            my.bad |= kStBadOffsets;
            continue;
        }
        const uint64_t m = b - a;
        if (m > (uint64_t)kMaxReadLen) {
            my.bad |= kStReadTooLong;
            continue;
        }
        int nn = 0;
        if ((int)m >= s) {
            nn = num_seeds > 0 ? num_seeds : (int)m / s;
            nn = min(nn, (int)m - s + 1);
        }
        if (nn > kMaxSeeds) my.bad |= kStTooManySeeds;
        nn *= stride;  // probe slots from here on (stride-k index)
        const int dm = dmax_per_read ? dmax_per_read[r] : d_max;
        if (dm < 0) my.bad |= kStBadDmax;
        const unsigned long long hh = (unsigned long long)nn * (unsigned long long)h_max;
        my.len = max(my.len, (unsigned int)m);
        my.L0 = max(my.L0, dm + c - 1);
        my.nseeds = max(my.nseeds, nn);
        my.hits = hh > my.hits ? hh : my.hits;
        my.light += (m <= (uint64_t)kLightBucketMaxM &&
                     nn <= (stride > 1 ? kLightVariantMaxSeeds : kLightBucketMaxSeeds) &&
                     dm + c - 1 <= kLightBucketMaxL);
        const int k = length_class(m);
#pragma unroll
        for (int q = 0; q < kClasses; ++q) {
            if (q != k) continue;
            my.c_n[q] += 1;
            my.c_len[q] = max(my.c_len[q], (unsigned int)m);
            my.c_L0[q] = max(my.c_L0[q], dm + c - 1);
            my.c_seeds[q] = max(my.c_seeds[q], nn);
            my.c_hits[q] = hh > my.c_hits[q] ? hh : my.c_hits[q];
        }
    }
    // warp partials in shared memory, merged by thread 0, then one atomic per field
    __shared__ StatsPart part[kStatsThreads / 32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        StatsPart other;
        other.bad = __shfl_xor_sync(kFull, my.bad, o);
        other.len = __shfl_xor_sync(kFull, my.len, o);
        other.L0 = __shfl_xor_sync(kFull, my.L0, o);
        other.nseeds = __shfl_xor_sync(kFull, my.nseeds, o);
        other.hits = __shfl_xor_sync(kFull, my.hits, o);
        other.light = __shfl_xor_sync(kFull, my.light, o);
#pragma unroll
        for (int q = 0; q < kClasses; ++q) {
            other.c_n[q] = __shfl_xor_sync(kFull, my.c_n[q], o);
            other.c_len[q] = __shfl_xor_sync(kFull, my.c_len[q], o);
            other.c_L0[q] = __shfl_xor_sync(kFull, my.c_L0[q], o);
            other.c_seeds[q] = __shfl_xor_sync(kFull, my.c_seeds[q], o);
            other.c_hits[q] = __shfl_xor_sync(kFull, my.c_hits[q], o);
        }
        stats_merge(my, other);
    }
    if (lane == 0) part[wib] = my;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) stats_merge(my, part[w]);
        if (my.bad) atomicOr(&st->status, my.bad);
        atomicMax(&st->max_len, my.len);
        atomicMax(&st->max_L0, my.L0);
        atomicMax(&st->max_seeds, my.nseeds);
        atomicMax(&st->max_hits_bound, my.hits);
        if (my.light) atomicAdd(&st->n_light, my.light);
#pragma unroll
        for (int q = 0; q < kClasses; ++q) {
            if (!my.c_n[q]) continue;
            atomicAdd(&st->cls_n[q], my.c_n[q]);
            atomicMax(&st->cls_max_len[q], my.c_len[q]);
            atomicMax(&st->cls_max_L0[q], my.c_L0[q]);
            atomicMax(&st->cls_max_seeds[q], my.c_seeds[q]);
            atomicMax(&st->cls_max_hits[q], my.c_hits[q]);
        }
        if (blockIdx.x == 0) {
            st->total_bases = offsets[n] - offsets[0];
            if (offsets[n] < offsets[0]) atomicOr(&st->status, kStBadOffsets);
        }
    }
}

// 16 ASCII bases (four little-endian 32-bit words) to one word of 2-bit codes;
// sets *bad when a byte is not one of A, C, G, T.  Four bases per operation:
// code = ((c >> 1) ^ (c >> 2)) & 3 on every byte at once (the shifted-in bits
// land above bit 1 of each byte and are masked off), the four 2-bit codes are
// gathered into one byte, and each byte is checked by rebuilding the letter of
// its code with a byte permutation of "ACGT" and comparing.
__device__ __forceinline__ uint32_t pack16_ascii(const uint32_t (&parts)[4], bool* bad) {
    uint32_t word = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t v = parts[q];
        const uint32_t t = ((v >> 1) ^ (v >> 2)) & 0x03030303u;  // code k at bits 8k, 8k+1
        const uint32_t u = t | (t >> 6);                          // codes 0,1 at bits 0-3; 2,3 at 16-19
        word |= ((u & 0xfu) | ((u >> 12) & 0xf0u)) << (8 * q);
        const uint32_t sel = (t & 3u) | ((t >> 4) & 0x30u) | ((t >> 8) & 0x300u) |
                             ((t >> 12) & 0x3000u);
        *bad |= __byte_perm(0x54474341u, 0u, sel) != v;  // 'A' 'C' 'G' 'T'
    }
    return word;
}

// Pack the concatenated reads (bytes [base, base + total) of `reads`) into
// 2-bit words, with kReadPadBases zero bases in front; flags non-ACGT bytes.
// Two independent words per thread and iteration keep two 16-byte loads in flight.
__global__ void k_pack_reads(const uint8_t* __restrict__ reads, uint64_t base, uint64_t total,
                             uint32_t* __restrict__ words, uint64_t nwords, int aligned16,
                             int* status) {
    constexpr uint64_t padw = kReadPadBases / 16;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (uint64_t w0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w0 < nwords;
         w0 += 2 * stride) {
        uint32_t parts[2][4];
        bool full[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const uint64_t w = w0 + u * stride;
            const uint64_t b0 = (w - padw) * 16;
            full[u] = w < nwords && w >= padw && b0 + 16 <= total && aligned16;
            if (full[u]) {
                const uint4 v = *reinterpret_cast<const uint4*>(reads + base + b0);
                parts[u][0] = v.x;
                parts[u][1] = v.y;
                parts[u][2] = v.z;
                parts[u][3] = v.w;
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const uint64_t w = w0 + u * stride;
            if (w >= nwords) continue;
            uint32_t word = 0;
            if (full[u]) {
                word = pack16_ascii(parts[u], &bad);
            } else if (w >= padw) {
                const uint64_t b0 = (w - padw) * 16;
                const uint8_t* src = reads + base + b0;
                for (uint64_t j = 0; j < 16 && b0 + j < total; ++j) {
                    const uint32_t ch = src[j];
                    bad |= !is_acgt(ch);
                    word |= code_of(ch) << (2 * j);
                }
            }
            words[w] = word;
        }
    }
    if (bad) atomicOr(status, kStBadBase);
}

// Distribute the reads the warp kernel must take (the thread-per-read kernel's
// leftovers, or all reads) into per-length-class lists (warp-aggregated atomics).
struct ClassLists {
    uint32_t* list;                     // class q at list + off[q]
    unsigned long long off[kClasses];
    unsigned long long* count;          // [kClasses]
};

__global__ void k_split_classes(const uint32_t* __restrict__ ids,
                                const unsigned long long* __restrict__ n_ids_dev, uint64_t n_all,
                                const uint64_t* __restrict__ offsets, ClassLists cl) {
    const uint64_t n_in = ids ? *n_ids_dev : n_all;
    const int lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t iters = (n_in + stride - 1) / stride;
    for (uint64_t it = 0; it < iters; ++it) {
        const uint64_t i = it * stride + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
        int k = -1;
        uint32_t r = 0;
        if (i < n_in) {
            r = ids ? ids[i] : (uint32_t)i;
            k = length_class(offsets[r + 1] - offsets[r]);
        }
#pragma unroll
        for (int q = 0; q < kClasses; ++q) {
            const unsigned mask = __ballot_sync(kFull, k == q);
            if (!mask) continue;
            unsigned long long base = 0;
            if (lane == __ffs(mask) - 1) base = atomicAdd(cl.count + q, (unsigned long long)__popc(mask));
            base = __shfl_sync(kFull, base, __ffs(mask) - 1);
            if (k == q) cl.list[cl.off[q] + base + __popc(mask & ((1u << lane) - 1))] = r;
        }
    }
}

// ---------------------------------------------------------------------------
// per-read candidate table (shared or global memory through generic pointers).
// The table is an open-addressing hash of (strand, p) keys sized for the read's
// seed hits; a dense list holds the slots in use, so picks and the clean-up
// after a read cost the number of distinct candidates, not the table size.
// Tables are left empty after every read.
// ---------------------------------------------------------------------------
__device__ __forceinline__ CandSlot empty_slot() {
    CandSlot e;
    e.key = kEmptyKey;
    e.votes = 0;
    e.state = kUnscored;
    return e;
}

// Adds one vote for key; returns the slot and whether the key is new.
__device__ __forceinline__ uint32_t table_add(CandSlot* tab, uint32_t mask, unsigned long long key,
                                              int* status, bool* inserted) {
    uint32_t h = (uint32_t)mix64(key) & mask;
    for (uint32_t step = 0; step <= mask; ++step) {
        const unsigned long long prev = atomicCAS(&tab[h].key, kEmptyKey, key);
        if (prev == kEmptyKey || prev == key) {
            atomicAdd(&tab[h].votes, 1u);
            *inserted = (prev == kEmptyKey);
            return h;
        }
        h = (h + 1) & mask;
    }
    atomicOr(status, kStTableFull);
    *inserted = false;
    return 0;
}

// most-voted unscored candidate, ties to the smaller key; 0 = none.
// packed = votes(11 bits) | (kKeyMask - key)(33 bits) | slot(20 bits)
__device__ __forceinline__ unsigned long long table_pick(const CandSlot* tab,
                                                         const uint32_t* dense, int nd, int lane) {
    unsigned long long best = 0;
    for (int j = lane; j < nd; j += 32) {
        const uint32_t slot = dense[j];
        const CandSlot c = tab[slot];
        if (c.state == kUnscored) {
            const unsigned long long v = ((unsigned long long)c.votes << 53) |
                                         ((kKeyMask - c.key) << 20) | (unsigned long long)slot;
            best = v > best ? v : best;
        }
    }
    return warp_max_u64(best);
}

// Initialise per-warp global candidate tables once after they are allocated.
__global__ void k_init_ctab(CandSlot* tab, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        tab[i] = empty_slot();
}

__device__ __forceinline__ unsigned long long bucket_of(unsigned long long key) {
    return ((key >> 6) << 1) | (key & 1);  // (strand, floor(p / 32))
}

struct FusedArgs {
    const uint32_t* genome;
    uint64_t G;
    int s;
    const IndexSlot* slots;
    uint64_t T;
    const uint32_t* positions;
    const uint32_t* rwords;
    const uint64_t* offsets;
    uint64_t base0;
    const uint32_t* order;  // processing order of read ids (NULL = identity)
    uint64_t n_items;
    const unsigned long long* n_items_dev;  // when set, the item count is read from here
    unsigned long long* head;
    int d_max, h_max, c, num_seeds;
    int first_seeds;  // non-popular seeds that vote before the first pick (<= 1: Algorithm 1)
    int collapse;     // share distances between identical windows in the parallel drain
    int stride;       // index stride: probes per seed
    const int32_t* dmax_per_read;
    uint8_t shifts[32];
    int n_shifts;
    snap_result* out;
    CandSlot* gtab;   // per-warp overflow tables, gcap slots each (kept empty)
    HitRec* ghits;    // per-warp overflow hit lists, gcap / 2 each
    uint32_t* gdense; // per-warp dense slot lists, gcap / 2 each
    uint32_t gcap;
    SeedRec* gseeds;  // per-warp seed records (seed_cap each) when not in shared memory
    uint32_t* gqbits; // per-warp q-gram bitmaps (2 x kQWords) for large limits, or NULL
    const SeedRec* hseeds;   // probe records of reads handed over by the thread-per-read
    const uint8_t* hprobed;  // kernel (kLightHandoverSlots per read), flagged per read
    // per read: its distinct candidates over all seeds (k_read_cost), which bounds
    // the table it needs, or kNoCount when not counted; NULL when not computed
    const uint32_t* read_nd;
    // when set, a read whose candidate table fits in no table this launch has is
    // listed here (defer_cap entries at most) instead of aligned; a later launch
    // aligns the listed reads (the allocation-free entry point)
    uint32_t* defer_ids;
    unsigned long long* defer_count;
    unsigned long long defer_cap;
    int* status;
    DevCounters* ctr;
    // per-warp shared-memory layout, in 32-bit words; every section offset is a
    // multiple of 4 words (16 bytes) because SeedRec / CandSlot / HitRec are
    // moved with 16-byte vector accesses
    int wx, wt, seed_cap, scap, lv_ints, warp_words;
    int off_xr, off_tw, off_seeds, off_tab, off_hits, off_dense, off_lv;
    int off_par;  // parallel-drain scratch (par_words(par_mmax) words), 0 = none
    int par_mmax;
};

struct WarpCounters {
    uint32_t seeds = 0, slot_reads = 0, list_entries = 0, ed_calls = 0, ed_over = 0;
    unsigned long long window_words = 0;
    uint32_t ed_filtered = 0, reads_done = 0, ed_collapsed = 0;
};

__device__ __forceinline__ void flush_counters(DevCounters* ctr, WarpCounters& c) {
    unsigned long long v[9] = {c.seeds, c.slot_reads, c.list_entries, c.ed_calls, c.ed_over,
                               c.window_words, c.ed_filtered, c.reads_done, c.ed_collapsed};
#pragma unroll
    for (int k = 0; k < 9; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(kFull, v[k], o);
    }
    if ((threadIdx.x & 31) == 0) {
        unsigned long long* dst = &ctr->seeds;
#pragma unroll
        for (int k = 0; k < 9; ++k)
            if (v[k]) atomicAdd(dst + k, v[k]);
    }
}

struct WarpMem {
    uint32_t* Xf;
    uint32_t* Xr;
    uint32_t* Tw;
    SeedRec* seeds;
    CandSlot* stab;
    HitRec* shits;
    uint32_t* sdense;
    int* lvA;
    int* lvB;
    CandSlot* gtab;
    HitRec* ghits;
    uint32_t* gdense;
    uint32_t* qbits;  // q-gram bitmaps of the read, one per strand (or NULL: no filter)
    int* job;         // team mode: the lead warp's posted job (see k_align_team)
    uint32_t* par;    // parallel-drain scratch, or NULL
};

// ---------------------------------------------------------------------------
// Parallel drain.  Once the Baeza-Yates test passes, Algorithm 1 scores every
// remaining candidate in pick order (most votes, then smaller key) with no
// early return, and the votes no longer change, so the whole drain order is
// known up front.  The warp ranks the unscored candidates once, then takes them
// 32 at a time: each lane computes one candidate's distance at a bound Lc with
// its own Landau-Vishkin (lv_lane), and the warp replays the 32 in order, each
// at the limit Algorithm 1 would use for it.  Every limit is d_best + c - 1,
// d_best - 1 or (d_best > d_max) d_max + c - 1, and d_best never grows, so
// Lc = min(d_best, d_max) + c - 1 bounds all later limits (a limit itself can
// grow: a new best in the old best's 32-base bucket can lift d_second clear of
// it).  A distance d0 found at Lc gives the one at L <= Lc as
// (d0 <= L ? d0 : over): the results are those of scoring one by one.
// ---------------------------------------------------------------------------
constexpr int kParMaxL = 7;                     // lane diagonals: 2 * 7 + 3 = 17
constexpr int kParMaxCands = 128;               // unscored candidates ranked at once
// scratch words per warp for reads up to mmax bases: the ranked keys, later the
// lanes' genome windows (column layout), then the slots in drain order and the
// lanes' diagonals
__host__ __device__ constexpr int par_window_words(int mmax) {
    return (15 + mmax + kParMaxL + 15) / 16 + 2;
}
__host__ __device__ constexpr int par_union_words(int mmax) {
    return 2 * kParMaxCands > 32 * par_window_words(mmax) ? 2 * kParMaxCands
                                                           : 32 * par_window_words(mmax);
}
// the lanes' diagonals are 16-bit (reads of the parallel drain are below 2^14 bases)
__host__ __device__ constexpr int par_words(int mmax) {
    return par_union_words(mmax) + kParMaxCands + (32 * (2 * kParMaxL + 3) + 1) / 2;
}

// ---------------------------------------------------------------------------
// q-gram rejection ahead of large-limit edit distances (the q-gram lemma).  If some prefix Y of
// the window W has Lev(X, Y) <= L, then X and Y share at least
// |X| - q + 1 - L*q q-grams (each edit touches at most q of X's q-grams, the
// others reappear in Y), and Y's q-grams are among W's.  Counting the window
// positions whose q-gram is in a bitmap of X's q-grams can only overcount that
// shared number, so a count below the bound proves the distance is over L and
// the rounds of the edit distance are skipped: the result is unchanged.
// ---------------------------------------------------------------------------
constexpr int kQ = 9;                          // q-gram length (18 bits: direct index)
constexpr int kQWords = (1 << (2 * kQ)) / 32;  // presence bitmap words per strand
constexpr int kQMinL = 48;                     // below this limit the rounds are cheap

// Whether the bound is tried: it must be able to fire (a positive bound), and
// the over-limit rounds it can save (about L^2 diagonal steps) must outweigh
// counting the window's m + L positions.
__host__ __device__ __forceinline__ bool use_qfilter(int m, int L) {
    return L >= kQMinL && (m - kQ + 1) - L * kQ > 0 && L * L >= 8 * (m + L);
}
constexpr uint32_t kQMask = (1u << (2 * kQ)) - 1u;

// Mark the q-grams of the packed sequence X (m bases) in bits (zero on entry).
__device__ __forceinline__ void build_qbits(const uint32_t* X, int m, uint32_t* bits, int lane) {
    for (int i = lane; i + kQ <= m; i += 32) {
        const uint32_t g = get16(X, (uint64_t)i) & kQMask;
        atomicOr(bits + (g >> 5), 1u << (g & 31));
    }
    __syncwarp();
}

// Zero the words build_qbits touched, leaving bits all zero again.
__device__ __forceinline__ void clear_qbits(const uint32_t* X, int m, uint32_t* bits, int lane) {
    __syncwarp();
    for (int i = lane; i + kQ <= m; i += 32) bits[(get16(X, (uint64_t)i) & kQMask) >> 5] = 0u;
    __syncwarp();
}

// Number of window positions whose q-gram is marked in bits.
__device__ __forceinline__ int count_qhits(const uint32_t* Tw, int tb, int n, const uint32_t* bits,
                                           int lane) {
    // several independent map loads in flight per lane (the map lives in L2)
    constexpr int kU = 4;
    const int npos = n - kQ + 1;
    int c = 0;
    for (int j0 = 0; j0 < npos; j0 += 32 * kU) {
        uint32_t word[kU], bit[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int j = j0 + u * 32 + lane;
            const uint32_t g = get16(Tw, (uint64_t)(tb + min(j, npos - 1))) & kQMask;
            bit[u] = j < npos ? (g & 31) : 32u;
            word[u] = __ldcg(bits + (g >> 5));
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) c += bit[u] < 32u ? (word[u] >> bit[u]) & 1u : 0u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    return c;
}

// Warp form of the bound for candidate (strand, window at tb of n bases): builds
// the strand's map on first use.
__device__ __forceinline__ bool qgram_rejects(const WarpMem& wm, int m, int strand, int tb, int n,
                                           int L, int lane, int& qbuilt) {
    uint32_t* bits = wm.qbits + strand * kQWords;
    if (!(qbuilt & (1 << strand))) {
        build_qbits(strand ? wm.Xr : wm.Xf, m, bits, lane);
        qbuilt |= 1 << strand;
    }
    return count_qhits(wm.Tw, tb, n, bits, lane) < (m - kQ + 1) - L * kQ;
}

// Per-thread share of count_qhits over positions tid, tid + nt, ... (no reduction).
__device__ __forceinline__ int count_qhits_part(const uint32_t* Tw, int tb, int n,
                                                const uint32_t* bits, int tid, int nt) {
    constexpr int kU = 4;
    const int npos = n - kQ + 1;
    int c = 0;
    for (int j0 = 0; j0 < npos; j0 += nt * kU) {
        uint32_t word[kU], bit[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int j = j0 + u * nt + tid;
            const uint32_t g = get16(Tw, (uint64_t)(tb + min(j, npos - 1))) & kQMask;
            bit[u] = j < npos ? (g & 31) : 32u;
            word[u] = __ldcg(bits + (g >> 5));
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) c += bit[u] < 32u ? (word[u] >> bit[u]) & 1u : 0u;
    }
    return c;
}

// ---------------------------------------------------------------------------
// Team mode.  When a length class has too few reads to fill the SMs with one
// warp per read, each block aligns one read at a time: its first warp (the
// lead) runs the per-read logic exactly as in warp mode, and every edit
// distance is computed by all warps of the block together.  The lead posts a
// job (op, key, limit, read length, which strands' q-gram maps are built) in
// shared memory and meets the helpers at a block barrier; all threads then run
// team_distance, whose result is uniform over the block.
// ---------------------------------------------------------------------------
constexpr int kTeamWarps = 8;
// team mode below max(8, longest read / 12) reads per SM: per-read work grows
// with the square of the limit, and one warp per read leaves long reads (and the
// slowest read of the class) latency-bound
constexpr int kTeamReadsPerSm = 8;
enum : int { kJobExit = 0, kJobDistance = 1 };
constexpr int kJobWords = 8;  // op, key lo, key hi, L, m, qbuilt, counter, pad

// Landau-Vishkin rounds over the whole block: diagonals of round e spread over
// all nt threads, one barrier per round (which also votes on completion).
__device__ inline int lv_team(const uint32_t* X, int m, const uint32_t* Tw, int tb, int n, int L,
                              int tid, int nt, int* Ra, int* Rb) {
    constexpr int NEG = -0x40000000;
    const int W = 2 * L + 3, off = L + 1;
    for (int i = tid; i < W; i += nt) {
        Ra[i] = NEG;
        Rb[i] = NEG;
    }
    __syncthreads();
    for (int e = 0; e <= L; ++e) {
        int done = 0;
        for (int idx = tid; idx < 2 * e + 1; idx += nt) {
            const int k = idx - e;
            int r;
            if (e == 0) {
                r = 0;
            } else {
                r = max(max(Ra[k + off] + 1, Ra[k + 1 + off] + 1), Ra[k - 1 + off]);
            }
            if (r > m) r = m;
            if (r + k > n) r = n - k;
            if (r < 0 || r + k < 0) {
                r = NEG;
            } else {
                r = slide(X, m, Tw, tb, n, r, k);
                done |= (r >= m);
            }
            Rb[k + off] = r;
        }
        if (__syncthreads_or(done)) return e;
        int* t = Ra;
        Ra = Rb;
        Rb = t;
    }
    return kOver;
}

// The distance job, run by every thread of the block with the same arguments.
// Returns the distance (kOver when over L) and sets *filtered when the q-gram
// bound decided it; builds the q-gram map of the candidate's strand if needed.
__device__ int team_distance(const FusedArgs& a, const WarpMem& wm, int m, unsigned long long key,
                             int L, int qbuilt, int tid, int nt, bool* filtered) {
    const uint64_t p = key >> 1;
    const int strand = (int)(key & 1);
    const uint64_t avail = a.G - p;
    const int n_t = (int)min(avail, (uint64_t)(m + L));
    const uint64_t w0 = p >> 4;
    const int tb = (int)(p & 15);
    const int nwt = (tb + n_t + 15) / 16 + 2;
    const uint32_t* X = strand ? wm.Xr : wm.Xf;
    for (int w = tid; w < nwt; w += nt) wm.Tw[w] = __ldg(a.genome + w0 + w);
    const int bound = (m - kQ + 1) - L * kQ;
    const bool use_q = wm.qbits && use_qfilter(m, L);
    uint32_t* bits = wm.qbits ? wm.qbits + strand * kQWords : nullptr;
    if (use_q && !(qbuilt & (1 << strand))) {
        for (int i = tid; i + kQ <= m; i += nt) {
            const uint32_t g = get16(X, (uint64_t)i) & kQMask;
            atomicOr(bits + (g >> 5), 1u << (g & 31));
        }
    }
    int* counter = wm.job + 6;
    if (tid == 0) *counter = 0;
    __syncthreads();
    *filtered = false;
    if (use_q) {
        int c = count_qhits_part(wm.Tw, tb, n_t, bits, tid, nt);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
        if ((tid & 31) == 0) atomicAdd(counter, c);
        __syncthreads();
        if (*counter < bound) {
            *filtered = true;
            return kOver;
        }
    }
    return lv_team(X, m, wm.Tw, tb, n_t, L, tid, nt, wm.lvA, wm.lvB);
}

// Helper warps of a team: run posted jobs until the lead posts kJobExit.
__device__ void team_helper(const FusedArgs& a, const WarpMem& wm) {
    for (;;) {
        __syncthreads();  // job posted
        const int op = wm.job[0];
        if (op == kJobExit) return;
        const unsigned long long key =
            (unsigned long long)(uint32_t)wm.job[1] | ((unsigned long long)(uint32_t)wm.job[2] << 32);
        const int L = wm.job[3], m = wm.job[4], qb = wm.job[5];
        bool filtered;
        team_distance(a, wm, m, key, L, qb, threadIdx.x, blockDim.x, &filtered);
    }
}

// ---------------------------------------------------------------------------
// Wave mode.  Team mode spreads one edit distance over the block, with a block
// barrier per diagonal round; when a class's reads carry many large-limit
// candidates the rounds are barrier- and latency-bound, and a read whose
// candidates are all near the limit holds one block for the whole tail of the
// launch.  Wave mode instead gives each warp of the block a candidate of its
// own.  Picks depend only on the votes, so the lead warp runs Algorithm 1 ahead
// of its scores: it adds seeds and picks (one pick per non-popular seed, as in
// the seed loop, or one per step of the drain) until it holds W picks, one per
// warp.  Every warp computes its pick's distance at Lb = min(d_best, dmax) + c - 1,
// which bounds every limit Algorithm 1 can use before those scores (d_best only
// falls; see the parallel drain), and the lead replays the steps in order, each
// score at its own limit with ED(L) = (d0 <= L ? d0 : over), and the exit tests
// after each seed.  When the Baeza-Yates test passes at a step before the last,
// the steps after it are undone (their seeds' votes taken back, their picks
// unscored again, candidates left without votes retired), so the drain starts
// from the state Algorithm 1 reaches there; an early return needs no undo.
// Results are those of scoring one candidate at a time.
// ---------------------------------------------------------------------------
constexpr int32_t kPending = -4;  // picked in the current wave, not yet replayed
constexpr int32_t kRetired = -3;  // no votes left after an undo: not a candidate
constexpr uint32_t kNoPick = 0xffffffffu;
constexpr int kWaveMaxWarps = 8;
// job words: op, picks, Lb, read length, then per pick its key (2 words) and result
constexpr int kWaveKeys = 4;
constexpr int kWaveRes = kWaveKeys + 2 * kWaveMaxWarps;
constexpr int kWaveJobWords = kWaveRes + kWaveMaxWarps + 4;
static_assert(kWaveJobWords % 4 == 0, "wave job words keep 16-byte alignment");

// Slot of a key that is in the table (kNoPick if it is not: cannot happen).
__device__ __forceinline__ uint32_t table_find(const CandSlot* tab, uint32_t mask,
                                               unsigned long long key) {
    uint32_t h = (uint32_t)mix64(key) & mask;
    for (uint32_t step = 0; step <= mask; ++step) {
        const unsigned long long k = tab[h].key;
        if (k == key) return h;
        if (k == kEmptyKey) break;
        h = (h + 1) & mask;
    }
    return kNoPick;
}

// One wave entry's distance by one warp: window staged in this warp's Tw, the
// q-gram bound (bits: the strand's map, built by the lead), then the rounds.
__device__ int wave_distance(const FusedArgs& a, const uint32_t* X, int m, unsigned long long key,
                             int L, uint32_t* Tw, int* lvA, int* lvB, const uint32_t* bits,
                             int lane, WarpCounters& wc) {
    const uint64_t p = key >> 1;
    const int n_t = (int)min(a.G - p, (uint64_t)(m + L));
    const uint64_t w0 = p >> 4;
    const int tb = (int)(p & 15);
    const int nwt = (tb + n_t + 15) / 16 + 2;
    for (int w = lane; w < nwt; w += 32) Tw[w] = __ldg(a.genome + w0 + w);
    __syncwarp();
    if (lane == 0) wc.window_words += (unsigned)nwt;
    if (bits && use_qfilter(m, L) &&
        count_qhits(Tw, tb, n_t, bits, lane) < (m - kQ + 1) - L * kQ) {
        if (lane == 0) wc.ed_filtered++;
        return kOver;
    }
    return lv_warp(X, m, Tw, tb, n_t, L, lane, lvA, lvB, a.status);
}

// Warp `g` > 0 of a wave block: its window and diagonal buffers follow the
// lead's layout; runs posted waves until the lead posts kJobExit.
__device__ void wave_helper(const FusedArgs& a, const WarpMem& wm, uint32_t* smem, int g,
                            WarpCounters& wc) {
    const int lane = threadIdx.x & 31;
    uint32_t* Tw = smem + a.warp_words + (size_t)(g - 1) * (a.wt + a.lv_ints);
    int* lvA = reinterpret_cast<int*>(Tw + a.wt);
    int* lvB = lvA + a.lv_ints / 2;
    for (;;) {
        __syncthreads();  // wave posted
        if (wm.job[0] == kJobExit) return;
        const int w = wm.job[1], Lb = wm.job[2], m = wm.job[3];
        if (g < w) {
            const unsigned long long key =
                (unsigned long long)(uint32_t)wm.job[kWaveKeys + 2 * g] |
                ((unsigned long long)(uint32_t)wm.job[kWaveKeys + 2 * g + 1] << 32);
            const int strand = (int)(key & 1);
            const uint32_t* bits = wm.qbits ? wm.qbits + strand * kQWords : nullptr;
            const int d = wave_distance(a, strand ? wm.Xr : wm.Xf, m, key, Lb, Tw, lvA, lvB, bits,
                                        lane, wc);
            if (lane == 0) wm.job[kWaveRes + g] = d;
        }
        __syncthreads();  // results in
    }
}

// Edit distance of candidate `key` at limit L (warp-wide, result uniform).  LVD
// selects the diagonal layout: D diagonals per lane in registers (L <= 32D/2 - 1),
// 0 for shared memory (any L), or -1 for shared memory behind the q-gram bound.
// One variant per kernel keeps the code small.
template <int LVD, bool TEAM>
__device__ __forceinline__ int candidate_distance(const FusedArgs& a, const WarpMem& wm, int m,
                                               unsigned long long key, int L, int lane,
                                               WarpCounters& wc, int& qbuilt) {
    if (L < 0) return kOver;
    if constexpr (TEAM) {
        // lead warp: post the job, then compute it with the helpers
        if (lane == 0) {
            wm.job[0] = kJobDistance;
            wm.job[1] = (int)(uint32_t)key;
            wm.job[2] = (int)(uint32_t)(key >> 32);
            wm.job[3] = L;
            wm.job[4] = m;
            wm.job[5] = qbuilt;
        }
        __syncthreads();  // job posted
        bool filtered;
        const int d = team_distance(a, wm, m, key, L, qbuilt, threadIdx.x, blockDim.x, &filtered);
        const int strand = (int)(key & 1);
        if (wm.qbits && use_qfilter(m, L)) qbuilt |= 1 << strand;
        if (lane == 0) {
            const uint64_t p = key >> 1;
            const int n_t = (int)min(a.G - p, (uint64_t)(m + L));
            wc.window_words += (unsigned)(((int)(p & 15) + n_t + 15) / 16 + 2);
            wc.ed_calls++;
            wc.ed_over += (d < 0);
            wc.ed_filtered += filtered;
        }
        __syncwarp();
        return d;
    }
    const uint64_t p = key >> 1;
    const int strand = (int)(key & 1);
    const uint64_t avail = a.G - p;
    const int n_t = (int)min(avail, (uint64_t)(m + L));
    const uint64_t w0 = p >> 4;
    const int tb = (int)(p & 15);
    const int nwt = (tb + n_t + 15) / 16 + 2;
    for (int w = lane; w < nwt; w += 32) wm.Tw[w] = __ldg(a.genome + w0 + w);
    __syncwarp();
    int d;
    if constexpr (LVD > 0) {
        d = lv_warp_reg<LVD>(strand ? wm.Xr : wm.Xf, m, wm.Tw, tb, n_t, L, lane);
    } else {
        bool rejected = false;
        if constexpr (LVD < 0)
            rejected = wm.qbits && use_qfilter(m, L) &&
                       qgram_rejects(wm, m, strand, tb, n_t, L, lane, qbuilt);
        if (rejected) {
            d = kOver;
            if (lane == 0) wc.ed_filtered++;
        } else {
            d = lv_warp(strand ? wm.Xr : wm.Xf, m, wm.Tw, tb, n_t, L, lane, wm.lvA, wm.lvB,
                        a.status);
        }
    }
    __syncwarp();
    if (lane == 0) {
        wc.window_words += (unsigned)nwt;
        wc.ed_calls++;
        wc.ed_over += (d < 0);
    }
    return d;
}

// VARIANT: the index has a stride > 1 or first_seeds > 1 (probe slots grouped
// per seed, picks deferred); without it a probe is a seed and every non-popular
// one picks.
// WAVE: the lead warp of a wave block (see wave_helper); with VARIANT false only.
template <int LVD, bool TEAM, bool VARIANT, bool WAVE = false>
__device__ __forceinline__ void align_one_read(const FusedArgs& a, const WarpMem& wm, uint64_t r,
                                               int lane, WarpCounters& wc) {
    static_assert(!(WAVE && (VARIANT || TEAM)), "wave mode: plain index, first_seeds <= 1");
    const uint64_t o0 = a.offsets[r], o1 = a.offsets[r + 1];
    const int m = (int)(o1 - o0);
    const uint64_t rb = o0 - a.base0 + kReadPadBases;
    const int s = a.s;
    int ng = 0;  // seeds
    if (m >= s) {
        ng = a.num_seeds > 0 ? a.num_seeds : m / s;
        ng = min(ng, m - s + 1);
    }
    const int stride = VARIANT ? a.stride : 1;
    const int n = ng * stride;  // probe slots (stride-k index: k per seed)
    const int dmax = a.dmax_per_read ? a.dmax_per_read[r] : a.d_max;
    const int c = a.c;
    long long res_loc = -1;
    int res_d = -1, res_strand = 0, res_cls = SNAP_NOT_FOUND;
    bool deferred = false;  // listed for a later launch (see FusedArgs::defer_ids)

    if (n > 0) {
        // ---- read and reverse complement, 2 bits per base ----
        const int nw = (m + 15) / 16;
        for (int w = lane; w < nw + 3; w += 32) {
            uint32_t f = 0, rc = 0;
            if (w < nw) {
                f = get16(a.rwords, rb + 16ull * w);
                rc = rev_groups32(~get16(a.rwords, rb + (uint64_t)m - 16 - 16ull * w));
            } else if (w == nw) {
                f = get16(a.rwords, rb + 16ull * w);  // tail of the last word (unused bases)
            }
            wm.Xf[w] = f;
            wm.Xr[w] = rc;
        }
        __syncwarp();
        // ---- seeds and index probes, one lane per probe ----
        unsigned int H = 0;
        int last_np = -1;  // last probe after which a pick happens (seeds-first variant)
        // a read the thread-per-read kernel probed before handing it over: its records
        const bool reuse = a.hprobed != nullptr && a.hprobed[r] != 0;
        if (reuse) {
            for (int i = lane; i < n; i += 32) {
                const SeedRec rec = a.hseeds[r * kLightHandoverSlots + i];
                wm.seeds[i] = rec;
                if ((rec.flags & (kSeedValid | kSeedPopular)) == kSeedValid) {
                    H += (unsigned int)rec.fwd_n + rec.rc_n;
                    if (VARIANT && (rec.flags & kSeedPick)) last_np = i;
                }
            }
        }
        for (int i = reuse ? n : lane; i < n; i += 32) {
            bool p0 = false;
            const int o = VARIANT ? probe_offset(i, stride, m, s, a.shifts, a.n_shifts, &p0)
                                  : seed_offset(i, m, s, a.shifts, a.n_shifts, &p0);
            SeedRec rec;
            rec.pad = 0;
            if (VARIANT && o < 0) {  // a probe that does not fit in the read
                rec.flags = 0;
                rec.offset = 0;
                rec.fwd_n = rec.rc_n = 0;
                rec.fwd_ref = rec.rc_ref = 0;
                wm.seeds[i] = rec;
                continue;
            }
            rec.flags = (uint8_t)(kSeedValid | (p0 ? kSeedPass0 : 0));
            rec.offset = (uint16_t)o;
            const uint64_t v = get32(wm.Xf, (uint64_t)o) & kmer_mask(s);
            uint32_t cnt = 0;
            lookup_seed(a.slots, a.T, a.positions, v, s, &rec, &cnt, a.status, &wc.slot_reads);
            wc.seeds++;
            if (cnt > (uint32_t)a.h_max) {
                rec.flags |= kSeedPopular;
            } else {
                H += (unsigned int)rec.fwd_n + rec.rc_n;
                if (stride == 1) {  // a probe is a seed
                    rec.flags |= (uint8_t)(kSeedPick | (p0 ? kSeedCountT : 0));
                    if (VARIANT) last_np = i;
                }
            }
            wm.seeds[i] = rec;
        }
        if (VARIANT && stride > 1 && !reuse) {  // per seed: its last non-popular probe picks
            __syncwarp();
            for (int g = lane; g < ng; g += 32)
                last_np = max(last_np, mark_seed_group(g, stride, n, [&](int i) {
                                  return &wm.seeds[i].flags;
                              }));
            __syncwarp();
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            H += __shfl_xor_sync(kFull, H, o);
            if (VARIANT) last_np = max(last_np, __shfl_xor_sync(kFull, last_np, o));
        }
        // ---- candidate table: shared memory when it fits, else this warp's global one ----
        // (sized for the distinct candidates when k_read_cost counted them, else
        // for every hit)
        uint32_t cap = 64;
        const uint32_t hb = (a.read_nd && a.read_nd[r] < H) ? a.read_nd[r] : H;
        while (cap < 2u * hb) cap <<= 1;
        CandSlot* tab;
        HitRec* hits;
        uint32_t* dense;
        bool ok = true;
        if (cap <= (uint32_t)a.scap) {
            tab = wm.stab;
            hits = wm.shits;
            dense = wm.sdense;
        } else if (wm.gtab && cap <= a.gcap) {
            tab = wm.gtab;
            hits = wm.ghits;
            dense = wm.gdense;
        } else {
            tab = nullptr;
            hits = nullptr;
            dense = nullptr;
            ok = false;
            if (a.defer_ids) {  // aligned by a later launch that has the tables
                deferred = true;
                if (lane == 0) {
                    const unsigned long long at = atomicAdd(a.defer_count, 1ull);
                    if (at < a.defer_cap)
                        a.defer_ids[at] = (uint32_t)r;
                    else
                        atomicOr(a.status, kStTableFull);
                }
            } else if (lane == 0) {
                atomicOr(a.status, kStTableFull);
            }
        }
        if (ok) {
            int nd = 0;        // distinct candidates so far (slots listed in dense)
            int qbuilt = 0;    // strands whose q-gram bitmap is built for this read
            int par_skip = 0;  // drain iterations before the parallel drain is retried
            int voted = 0;     // non-popular seeds whose votes are in
            int d_best = kInf, d_second = kInf, nh = 0, t = 0;
            unsigned long long best_key = 0;
            bool any_nonpopular = false, returned = false;

            auto limit = [&]() -> int {
                if (d_best > dmax) return dmax + c - 1;
                if (d_second >= d_best + c) return d_best + c - 1;
                return d_best - 1;
            };
            // the bookkeeping of one scored candidate (warp-uniform arguments)
            auto record = [&](uint32_t slot, unsigned long long key, int d) {
                if (lane == 0) {
                    tab[slot].state = d >= 0 ? d : kOver;
                    if (d >= 0) {
                        HitRec h;
                        h.key = key;
                        h.d = d;
                        h.pad = 0;
                        hits[nh] = h;
                    }
                }
                __syncwarp();
                if (d >= 0) {
                    ++nh;
                    if (d < d_best) {
                        d_best = d;
                        best_key = key;
                        const unsigned long long bb = bucket_of(key);
                        int v = kInf;
                        for (int j = lane; j < nh; j += 32) {
                            const HitRec h = hits[j];
                            if (bucket_of(h.key) != bb) v = min(v, h.d);
                        }
                        d_second = warp_min_i32(v);
                    } else if (bucket_of(key) != bucket_of(best_key)) {
                        d_second = min(d_second, d);
                    }
                }
            };
            auto score = [&](unsigned long long packed) {
                const uint32_t slot = (uint32_t)(packed & 0xfffffu);
                const unsigned long long key = kKeyMask - ((packed >> 20) & kKeyMask);
                const int L = limit();
                const int d = candidate_distance<LVD, TEAM>(a, wm, m, key, L, lane, wc, qbuilt);
                record(slot, key, d);
            };
            // the whole drain, in parallel (see par_words); false when it does not
            // apply (limit above kParMaxL or too many candidates) and nothing was done
            auto drain_parallel = [&]() -> bool {
                if (min(d_best, dmax) + c - 1 > kParMaxL) return false;
                unsigned long long* upk = reinterpret_cast<unsigned long long*>(wm.par);
                uint32_t* Tp = wm.par;  // after ranking: the lanes' windows
                uint32_t* order = wm.par + par_union_words(a.par_mmax);
                int16_t* Rp = reinterpret_cast<int16_t*>(order + kParMaxCands);
                // unscored candidates, packed as in table_pick (distinct keys)
                int U = 0;
                for (int j0 = 0; j0 < nd; j0 += 32) {
                    const int j = j0 + lane;
                    unsigned long long pk = 0;
                    if (j < nd) {
                        const uint32_t slot = dense[j];
                        const CandSlot cs = tab[slot];
                        if (cs.state == kUnscored)
                            pk = ((unsigned long long)cs.votes << 53) |
                                 ((kKeyMask - cs.key) << 20) | (unsigned long long)slot;
                    }
                    const unsigned b = __ballot_sync(kFull, pk != 0);
                    const int pos = U + __popc(b & ((1u << lane) - 1));
                    if (pk && pos < kParMaxCands) upk[pos] = pk;
                    U += __popc(b);
                }
                if (U > kParMaxCands) {
                    par_skip = U - kParMaxCands;  // sequential picks until few enough are left
                    return false;
                }
                __syncwarp();
                // drain order: entry e goes to position #{i : upk[i] > upk[e]}
                for (int e = lane; e < U; e += 32) {
                    const unsigned long long mine = upk[e];
                    int rank = 0;
                    for (int i = 0; i < U; ++i) rank += (upk[i] > mine);
                    order[rank] = (uint32_t)(mine & 0xfffffu);
                }
                __syncwarp();  // upk is reused for the windows
                // chunks of 32 in pick order
                for (int c0 = 0; c0 < U; c0 += 32) {
                    const int k = min(32, U - c0);
                    const uint32_t* chunk = order + c0;
                    const int Lc = min(d_best, dmax) + c - 1;  // bounds every later limit
                    int d0 = kOver;
                    unsigned words = 0;
                    unsigned long long my_key = 0;
                    bool staged = false;  // this lane's window is in Tp
                    int my_tb = 0, my_n = 0;
                    if (lane < k) {
                        my_key = tab[chunk[lane]].key;
                        if (Lc >= 0) {
                            const uint64_t p = my_key >> 1;
                            const int n_t = (int)min(a.G - p, (uint64_t)(m + Lc));
                            const int tb = (int)(p & 15);
                            const int nwt = (tb + n_t + 15) / 16 + 2;
                            if (nwt <= par_window_words(a.par_mmax)) {
                                const uint32_t* gw = a.genome + (p >> 4);
                                for (int w = 0; w < nwt; ++w) Tp[w * 32 + lane] = __ldg(gw + w);
                                words = (unsigned)nwt;
                                staged = true;
                                my_tb = tb;
                                my_n = n_t;
                            } else {
                                atomicOr(a.status, kStInternal);  // cannot happen: layout bug
                            }
                        }
                    }
                    // exact-duplicate collapsing: a lane whose window equals, base for
                    // base and on the same strand, that of a lower lane of the chunk
                    // takes that lane's distance instead of computing its own
                    int leader = lane;
                    if (a.collapse) {
                        __syncwarp();
                        uint64_t h = 0;
                        if (staged) {
                            h = mix64((uint64_t)my_n * 2 + (my_key & 1));
                            for (int b = 0; b < my_n; b += 16) {
                                uint32_t x = get16s(Tp + lane, my_tb + b, 32);
                                if (my_n - b < 16) x &= (1u << (2 * (my_n - b))) - 1u;
                                h = mix64(h ^ x);
                            }
                        }
                        const int my_sn = staged ? 2 * my_n + (int)(my_key & 1) + 1 : 0;
                        for (int q = 0; q < 32; ++q) {
                            const uint64_t hq = __shfl_sync(kFull, h, q);
                            const int snq = __shfl_sync(kFull, my_sn, q);  // length, strand
                            const int tq = __shfl_sync(kFull, my_tb, q);
                            if (staged && leader == lane && q < lane && snq == my_sn && hq == h) {
                                // same hash: compare the two windows exactly
                                bool same = true;
                                for (int b = 0; b < my_n && same; b += 16) {
                                    uint32_t x = get16s(Tp + lane, my_tb + b, 32) ^
                                                 get16s(Tp + q, tq + b, 32);
                                    if (my_n - b < 16) x &= (1u << (2 * (my_n - b))) - 1u;
                                    same = x == 0;
                                }
                                if (same) leader = q;
                            }
                        }
                    }
                    if (staged && leader == lane)
                        d0 = lv_lane((my_key & 1) ? wm.Xr : wm.Xf, 1, m, Tp + lane, 32, my_tb,
                                     my_n, Lc, Rp + lane, 32);
                    if (a.collapse) {
                        const int dl = __shfl_sync(kFull, d0, leader);
                        if (leader != lane) {
                            d0 = dl;
                            wc.ed_collapsed++;
                        }
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) words += __shfl_xor_sync(kFull, words, o);
                    if (lane == 0) wc.window_words += words;
                    // a candidate over Lc is over at its own limit and changes nothing
                    // but its state (written by its lane); only those within Lc are
                    // replayed in order, each at the limit of its turn, and the ones
                    // between them are counted at the limit they share
                    const unsigned within = __ballot_sync(kFull, lane < k && d0 >= 0);
                    if (lane < k && d0 < 0) tab[chunk[lane]].state = kOver;
                    int next = 0;  // first position of the chunk not counted yet
                    for (unsigned mm = within;; mm &= mm - 1) {
                        const int j = mm ? __ffs(mm) - 1 : k;
                        const int L = limit();
                        if (L >= 0 && lane == 0) {
                            wc.ed_calls += (uint32_t)(j - next);
                            wc.ed_over += (uint32_t)(j - next);
                        }
                        if (!mm) break;
                        const unsigned long long key = __shfl_sync(kFull, my_key, j);
                        const int dj = __shfl_sync(kFull, d0, j);
                        const int d = (L >= 0 && dj <= L) ? dj : kOver;
                        if (L >= 0 && lane == 0) {
                            wc.ed_calls++;
                            wc.ed_over += (d < 0);
                        }
                        record(chunk[j], key, d);
                        next = j + 1;
                    }
                }
                return true;
            };

            if constexpr (WAVE) {
            // Wave mode (see wave_helper): steps of Algorithm 1 taken ahead of their
            // scores, W picks at a time, then replayed in order.
            const int W = (int)(blockDim.x >> 5);
            // the votes of seed record `rec`: added (new candidates listed in
            // dense), or taken back (undo = true) after a drain started earlier
            auto seed_votes = [&](const SeedRec& rec, bool undo) {
                const int o = rec.offset;
                const int tot = (int)rec.fwd_n + rec.rc_n;
                for (int j0 = 0; j0 < tot; j0 += 32) {
                    const int j = j0 + lane;
                    bool ins = false;
                    uint32_t slot = 0;
                    if (j < tot) {
                        const bool fwd = j < rec.fwd_n;
                        uint32_t l;
                        if (fwd) {
                            l = (rec.flags & kSeedFwdInline)
                                    ? rec.fwd_ref : __ldg(a.positions + rec.fwd_ref + j);
                        } else {
                            const int jj = j - rec.fwd_n;
                            l = (rec.flags & kSeedRcInline)
                                    ? rec.rc_ref : __ldg(a.positions + rec.rc_ref + jj);
                        }
                        const long long p = fwd ? (long long)l - o : (long long)l - (m - o - s);
                        if (p >= 0) {
                            const unsigned long long key =
                                2ull * (unsigned long long)p + (fwd ? 0 : 1);
                            if (undo) {
                                const uint32_t sl = table_find(tab, cap - 1, key);
                                if (sl != kNoPick)
                                    atomicSub(&tab[sl].votes, 1u);
                                else
                                    atomicOr(a.status, kStInternal);  // cannot happen
                            } else {
                                wc.list_entries += (rec.flags & kSeedFwdInline) ? 0u : 1u;
                                slot = table_add(tab, cap - 1, key, a.status, &ins);
                            }
                        }
                    }
                    if (!undo) {
                        const unsigned nb = __ballot_sync(kFull, ins);
                        if (ins) dense[nd + __popc(nb & ((1u << lane) - 1))] = slot;
                        nd += __popc(nb);
                    }
                }
                __syncwarp();
            };
            bool draining = false;
            int i = 0;
            for (;;) {
                // ---- build: one step per non-popular seed (in the drain, per pick) ----
                const int Lb = min(d_best, dmax) + c - 1;  // bounds every limit below
                int w = 0, ns = 0;
                uint32_t st_slot = kNoPick;  // step `lane`: its pick (or none), t and i after it
                unsigned long long st_key = 0;
                int st_t = 0, st_i = 0;
                bool seeds_over = false;
                while (w < W && ns < 32) {
                    if (!draining) {
                        while (i < n && (wm.seeds[i].flags & kSeedPopular) != 0) ++i;
                        if (i >= n) {
                            seeds_over = true;
                            break;
                        }
                        const SeedRec rec = wm.seeds[i++];
                        any_nonpopular = true;
                        seed_votes(rec, false);
                        if (rec.flags & kSeedCountT) ++t;
                    }
                    const unsigned long long pk = table_pick(tab, dense, nd, lane);
                    if (!pk && draining) break;  // the drain has scored everything
                    uint32_t slot = kNoPick;
                    unsigned long long key = 0;
                    if (pk) {
                        slot = (uint32_t)(pk & 0xfffffu);
                        key = kKeyMask - ((pk >> 20) & kKeyMask);
                        if (lane == 0) {
                            tab[slot].state = kPending;
                            wm.job[kWaveKeys + 2 * w] = (int)(uint32_t)key;
                            wm.job[kWaveKeys + 2 * w + 1] = (int)(uint32_t)(key >> 32);
                        }
                        ++w;
                    }
                    if (lane == ns) {
                        st_slot = slot;
                        st_key = key;
                        st_t = t;
                        st_i = i;
                    }
                    ++ns;
                    __syncwarp();
                }
                if (ns == 0) break;  // seeds used up, or the drain is over
                // ---- the wave's distances at Lb, one warp each ----
                if (w > 0 && Lb >= 0) {
                    // q-gram maps of the strands this wave needs, before any warp counts
                    if (wm.qbits && use_qfilter(m, Lb)) {
                        int need = 0;
                        for (int e = 0; e < w; ++e)
                            need |= 1 << (wm.job[kWaveKeys + 2 * e] & 1);
                        for (int sd = 0; sd < 2; ++sd) {
                            if ((need >> sd) & 1 && !(qbuilt & (1 << sd))) {
                                build_qbits(sd ? wm.Xr : wm.Xf, m, wm.qbits + sd * kQWords, lane);
                                qbuilt |= 1 << sd;
                            }
                        }
                    }
                    if (lane == 0) {
                        wm.job[0] = kJobDistance;
                        wm.job[1] = w;
                        wm.job[2] = Lb;
                        wm.job[3] = m;
                    }
                    __syncthreads();  // wave posted
                    const unsigned long long key0 =
                        (unsigned long long)(uint32_t)wm.job[kWaveKeys] |
                        ((unsigned long long)(uint32_t)wm.job[kWaveKeys + 1] << 32);
                    const int sd0 = (int)(key0 & 1);
                    const int d0 = wave_distance(a, sd0 ? wm.Xr : wm.Xf, m, key0, Lb, wm.Tw, wm.lvA,
                                                 wm.lvB, wm.qbits ? wm.qbits + sd0 * kQWords : nullptr,
                                                 lane, wc);
                    if (lane == 0) wm.job[kWaveRes] = d0;
                    __syncthreads();  // results in
                }
                // ---- replay the steps in order ----
                bool stop = false;
                int e = 0;  // wave entry of the next pick
                for (int sx = 0; sx < ns; ++sx) {
                    const uint32_t slot = __shfl_sync(kFull, st_slot, sx);
                    const unsigned long long key = __shfl_sync(kFull, st_key, sx);
                    const int ts = __shfl_sync(kFull, st_t, sx);
                    const int is = __shfl_sync(kFull, st_i, sx);
                    if (slot != kNoPick) {
                        const int L = limit();
                        int d = kOver;
                        if (L >= 0) {
                            if (L > Lb && lane == 0) atomicOr(a.status, kStInternal);  // cannot happen
                            const int dw = Lb >= 0 ? wm.job[kWaveRes + e] : kOver;
                            d = (dw >= 0 && dw <= L) ? dw : kOver;
                            if (lane == 0) {
                                wc.ed_calls++;
                                wc.ed_over += (d < 0);
                            }
                        }
                        record(slot, key, d);
                        ++e;
                    }
                    if (draining) continue;
                    if (d_best < c && d_second < d_best + c) {
                        returned = true;
                        stop = true;
                        break;
                    }
                    if (ts >= d_best + c) {
                        draining = true;
                        if (sx + 1 < ns) {
                            // undo the later steps: picks unscored again, votes taken back
                            for (int sy = sx + 1; sy < ns; ++sy) {
                                const uint32_t sl = __shfl_sync(kFull, st_slot, sy);
                                const int iy = __shfl_sync(kFull, st_i, sy);
                                if (sl != kNoPick && lane == 0) tab[sl].state = kUnscored;
                                __syncwarp();
                                seed_votes(wm.seeds[iy - 1], true);
                            }
                            // candidates with no votes left do not exist at this step
                            for (int j = lane; j < nd; j += 32) {
                                const uint32_t sl = dense[j];
                                if (tab[sl].votes == 0 && tab[sl].state == kUnscored)
                                    tab[sl].state = kRetired;
                            }
                            __syncwarp();
                            t = ts;
                            i = is;
                        }
                        break;
                    }
                }
                if (stop) break;
                if (seeds_over && !draining) break;  // Algorithm 1's seed loop is over
            }
            } else {
            // One pass per non-popular seed: add its votes, pick and score one
            // candidate, test the exits.  Once the Baeza-Yates test passes the loop
            // only picks and scores (no early return) until nothing is left.
            bool draining = false;
            int i = 0;
            for (;;) {
                if constexpr (LVD > 0 && !TEAM) {
                    if (draining && wm.par) {
                        if (par_skip == 0 && drain_parallel()) break;
                        par_skip = max(0, par_skip - 1);
                    }
                }
                SeedRec rec;
                if (!draining) {
                    while (i < n && (VARIANT ? (wm.seeds[i].flags & (kSeedValid | kSeedPopular)) !=
                                                   kSeedValid
                                             : (wm.seeds[i].flags & kSeedPopular) != 0))
                        ++i;
                    if (i >= n) break;
                    rec = wm.seeds[i++];
                    any_nonpopular = true;
                const int o = rec.offset;
                const int tot = (int)rec.fwd_n + rec.rc_n;
                for (int j0 = 0; j0 < tot; j0 += 32) {
                    const int j = j0 + lane;
                    bool ins = false;
                    uint32_t slot = 0;
                    if (j < tot) {
                        const bool fwd = j < rec.fwd_n;
                        uint32_t l;
                        if (fwd) {
                            l = (rec.flags & kSeedFwdInline)
                                    ? rec.fwd_ref : __ldg(a.positions + rec.fwd_ref + j);
                        } else {
                            const int jj = j - rec.fwd_n;
                            l = (rec.flags & kSeedRcInline)
                                    ? rec.rc_ref : __ldg(a.positions + rec.rc_ref + jj);
                        }
                        wc.list_entries += (rec.flags & kSeedFwdInline) ? 0u : 1u;
                        const long long p = fwd ? (long long)l - o : (long long)l - (m - o - s);
                        if (p >= 0)
                            slot = table_add(tab, cap - 1,
                                             2ull * (unsigned long long)p + (fwd ? 0 : 1),
                                             a.status, &ins);
                    }
                    const unsigned nb = __ballot_sync(kFull, ins);
                    if (ins) dense[nd + __popc(nb & ((1u << lane) - 1))] = slot;
                    nd += __popc(nb);
                }
                __syncwarp();
                if (rec.flags & kSeedCountT) ++t;
                if constexpr (VARIANT) {
                    if (!(rec.flags & kSeedPick)) continue;  // more probes of this seed to come
                    // seeds-first variant: the first first_seeds non-popular seeds (all
                    // of them when fewer remain) vote before the first pick; no exit
                    // test can pass before a score
                    if (++voted < a.first_seeds && i <= last_np) continue;
                }
                }
                const unsigned long long pk = table_pick(tab, dense, nd, lane);
                if (pk) {
                    score(pk);
                } else if (draining) {
                    break;
                }
                if (!draining) {
                    if (d_best < c && d_second < d_best + c) {
                        returned = true;
                        break;
                    }
                    if (t >= d_best + c) draining = true;
                }
            }
            }  // WAVE
            const bool all_popular = !any_nonpopular;  // n >= 1 here
            if (!returned && d_best <= dmax && d_second >= d_best + c) {
                res_cls = SNAP_SINGLE_HIT;
            } else if (returned || d_best <= dmax || all_popular) {
                res_cls = SNAP_MULTIPLE_HITS;
            } else {
                res_cls = SNAP_NOT_FOUND;
            }
            if (res_cls != SNAP_NOT_FOUND && d_best <= dmax) {
                res_loc = (long long)(best_key >> 1);
                res_strand = (int)(best_key & 1);
                res_d = d_best;
            }
            // leave the table and the q-gram maps empty for the next read
            __syncwarp();
            for (int j = lane; j < nd; j += 32) tab[dense[j]] = empty_slot();
            if (qbuilt & 1) clear_qbits(wm.Xf, m, wm.qbits, lane);
            if (qbuilt & 2) clear_qbits(wm.Xr, m, wm.qbits + kQWords, lane);
            __syncwarp();
        }
    }
    if (lane == 0 && !deferred) {
        wc.reads_done++;
        // two 8-byte stores: snap_result arrays need only their natural alignment
        unsigned long long* dst = reinterpret_cast<unsigned long long*>(a.out + r);
        dst[0] = (unsigned long long)res_loc;
        dst[1] = (unsigned long long)(uint32_t)res_d |
                 ((unsigned long long)((uint32_t)res_strand | ((uint32_t)res_cls << 8)) << 32);
    }
    __syncwarp();
}

template <int LVD, bool VARIANT>
__global__ void __launch_bounds__(256, 4) k_align_fused(FusedArgs a) {
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t* base = smem + (size_t)wib * a.warp_words;
    WarpMem wm;
    wm.Xf = base;
    wm.Xr = base + a.off_xr;
    wm.Tw = base + a.off_tw;
    wm.seeds = a.gseeds ? a.gseeds + ((uint64_t)blockIdx.x * (blockDim.x >> 5) + wib) * a.seed_cap
                        : reinterpret_cast<SeedRec*>(base + a.off_seeds);
    wm.stab = reinterpret_cast<CandSlot*>(base + a.off_tab);
    wm.shits = reinterpret_cast<HitRec*>(base + a.off_hits);
    wm.sdense = base + a.off_dense;
    wm.lvA = a.lv_ints ? reinterpret_cast<int*>(base + a.off_lv) : nullptr;
    wm.lvB = a.lv_ints ? wm.lvA + a.lv_ints / 2 : nullptr;
    const uint64_t gw = (uint64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    wm.gtab = a.gtab ? a.gtab + gw * a.gcap : nullptr;
    wm.ghits = a.ghits ? a.ghits + gw * (a.gcap / 2) : nullptr;
    wm.gdense = a.gdense ? a.gdense + gw * (a.gcap / 2) : nullptr;
    wm.qbits = a.gqbits ? a.gqbits + gw * (2 * kQWords) : nullptr;
    wm.par = a.off_par ? base + a.off_par : nullptr;
    for (int j = lane; j < a.scap; j += 32) wm.stab[j] = empty_slot();
    __syncwarp();
    WarpCounters wc;
    const unsigned long long n_items = a.n_items_dev ? *a.n_items_dev : a.n_items;
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(a.head, 1ull);
        it = __shfl_sync(kFull, it, 0);
        if (it >= n_items) break;
        const uint64_t r = a.order ? a.order[it] : it;
        align_one_read<LVD, false, VARIANT>(a, wm, r, lane, wc);
    }
    flush_counters(a.ctr, wc);
}

// Team mode (see team_distance): one read per block at a time, kTeamWarps warps;
// warp 0 leads, the shared-memory layout is that of one warp plus the job words.
template <bool VARIANT>
__global__ void __launch_bounds__(kTeamWarps * 32) k_align_team(FusedArgs a) {
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    WarpMem wm;
    wm.Xf = smem;
    wm.Xr = smem + a.off_xr;
    wm.Tw = smem + a.off_tw;
    wm.seeds = a.gseeds ? a.gseeds + (uint64_t)blockIdx.x * a.seed_cap
                        : reinterpret_cast<SeedRec*>(smem + a.off_seeds);
    wm.stab = reinterpret_cast<CandSlot*>(smem + a.off_tab);
    wm.shits = reinterpret_cast<HitRec*>(smem + a.off_hits);
    wm.sdense = smem + a.off_dense;
    wm.lvA = reinterpret_cast<int*>(smem + a.off_lv);
    wm.lvB = wm.lvA + a.lv_ints / 2;
    const uint64_t gw = blockIdx.x;
    wm.gtab = a.gtab ? a.gtab + gw * a.gcap : nullptr;
    wm.ghits = a.ghits ? a.ghits + gw * (a.gcap / 2) : nullptr;
    wm.gdense = a.gdense ? a.gdense + gw * (a.gcap / 2) : nullptr;
    wm.qbits = a.gqbits ? a.gqbits + gw * (2 * kQWords) : nullptr;
    wm.job = reinterpret_cast<int*>(smem + a.warp_words);
    wm.par = nullptr;
    if (wib != 0) {
        team_helper(a, wm);
        return;
    }
    for (int j = lane; j < a.scap; j += 32) wm.stab[j] = empty_slot();
    __syncwarp();
    WarpCounters wc;
    const unsigned long long n_items = a.n_items_dev ? *a.n_items_dev : a.n_items;
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(a.head, 1ull);
        it = __shfl_sync(kFull, it, 0);
        if (it >= n_items) break;
        const uint64_t r = a.order ? a.order[it] : it;
        align_one_read<0, true, VARIANT>(a, wm, r, lane, wc);
    }
    if (lane == 0) wm.job[0] = kJobExit;
    __syncthreads();  // releases the helpers
    flush_counters(a.ctr, wc);
}

// Wave mode (see wave_helper): one read per block at a time, blockDim.x / 32
// warps (2 to 8), each with its own window and diagonal buffers after the lead's
// layout, then the job words.  Plain index and first_seeds <= 1 only.
__global__ void __launch_bounds__(kWaveMaxWarps * 32) k_align_wave(FusedArgs a) {
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int W = (int)(blockDim.x >> 5);
    WarpMem wm;
    wm.Xf = smem;
    wm.Xr = smem + a.off_xr;
    wm.Tw = smem + a.off_tw;
    wm.seeds = a.gseeds ? a.gseeds + (uint64_t)blockIdx.x * a.seed_cap
                        : reinterpret_cast<SeedRec*>(smem + a.off_seeds);
    wm.stab = reinterpret_cast<CandSlot*>(smem + a.off_tab);
    wm.shits = reinterpret_cast<HitRec*>(smem + a.off_hits);
    wm.sdense = smem + a.off_dense;
    wm.lvA = reinterpret_cast<int*>(smem + a.off_lv);
    wm.lvB = wm.lvA + a.lv_ints / 2;
    const uint64_t gw = blockIdx.x;
    wm.gtab = a.gtab ? a.gtab + gw * a.gcap : nullptr;
    wm.ghits = a.ghits ? a.ghits + gw * (a.gcap / 2) : nullptr;
    wm.gdense = a.gdense ? a.gdense + gw * (a.gcap / 2) : nullptr;
    wm.qbits = a.gqbits ? a.gqbits + gw * (2 * kQWords) : nullptr;
    wm.job = reinterpret_cast<int*>(smem + a.warp_words + (size_t)(W - 1) * (a.wt + a.lv_ints));
    wm.par = nullptr;
    WarpCounters wc;
    if (wib != 0) {
        wave_helper(a, wm, smem, wib, wc);
        flush_counters(a.ctr, wc);
        return;
    }
    for (int j = lane; j < a.scap; j += 32) wm.stab[j] = empty_slot();
    __syncwarp();
    const unsigned long long n_items = a.n_items_dev ? *a.n_items_dev : a.n_items;
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(a.head, 1ull);
        it = __shfl_sync(kFull, it, 0);
        if (it >= n_items) break;
        const uint64_t r = a.order ? a.order[it] : it;
        align_one_read<0, false, false, true>(a, wm, r, lane, wc);
    }
    if (lane == 0) wm.job[0] = kJobExit;
    __syncthreads();  // releases the helpers
    flush_counters(a.ctr, wc);
}

// ---------------------------------------------------------------------------
// Read order of a block-per-read class.  A block aligns one read at a time and
// a read's cost grows with the candidates Algorithm 1 scores (one pick per
// non-popular seed while unscored candidates remain), so a few repeat-rich
// reads can outlast the rest of the launch.  k_read_cost estimates each read's
// picks as min(non-popular seeds, distinct candidates over all seeds) from its
// probes alone, and k_order_by_cost lists the class's reads by that estimate,
// largest first (longest-processing-time order).  The distinct count also
// bounds the read's candidate table, which then often fits in shared memory
// where its hit count does not.  Results do not depend on either.
// ---------------------------------------------------------------------------
constexpr int kCostWarps = 4;
constexpr int kCostSlots = 1024;  // per-warp key set; counting stops past half of it
constexpr uint32_t kNoCount = 0xffffffffu;
constexpr int kCostBuckets = 1024;

struct CostArgs {
    const uint64_t* offsets;
    uint64_t n;
    const uint32_t* rwords;
    uint64_t base0;
    int s, num_seeds, h_max;
    uint8_t shifts[32];
    int n_shifts;
    const IndexSlot* slots;
    uint64_t T;
    const uint32_t* positions;
    int* status;
    unsigned mask;     // length classes whose reads are counted
    unsigned len_mask; // length classes whose reads are keyed by length alone (m / 4)
    uint32_t* cost;    // per read: min(non-popular seeds, distinct candidates, buckets - 1)
    uint32_t* read_nd; // per read: distinct candidates, or kNoCount past kCostSlots / 2
    unsigned* need;    // per class: the largest table need (distinct count, else hits)
};

// One warp per read of the batch whose length class is in `mask`.
__global__ void __launch_bounds__(kCostWarps * 32) k_read_cost(CostArgs a) {
    __shared__ unsigned long long sets[kCostWarps * kCostSlots];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned long long* hs = sets + wib * kCostSlots;
    for (int j = lane; j < kCostSlots; j += 32) hs[j] = kEmptyKey;
    __syncwarp();
    uint32_t steps = 0;
    for (uint64_t r = (uint64_t)blockIdx.x * kCostWarps + wib; r < a.n;
         r += (uint64_t)gridDim.x * kCostWarps) {
        const uint64_t o0 = a.offsets[r];
        const int m = (int)(a.offsets[r + 1] - o0);
        const int q = length_class((uint64_t)m);
        if ((a.len_mask >> q) & 1u) {
            if (lane == 0) a.cost[r] = (uint32_t)min(m >> 2, kCostBuckets - 1);
            continue;
        }
        if (!((a.mask >> q) & 1u)) continue;
        const uint64_t rb = o0 - a.base0 + kReadPadBases;
        const int s = a.s;
        int ng = 0;
        if (m >= s) {
            ng = a.num_seeds > 0 ? a.num_seeds : m / s;
            ng = min(ng, m - s + 1);
        }
        int nnp = 0, nd = 0;
        unsigned H = 0;  // hits of the non-popular seeds, as the align kernels count them
        bool full = false;
        for (int i0 = 0; i0 < ng; i0 += 32) {
            const int i = i0 + lane;
            SeedRec rec;
            rec.flags = 0;
            rec.fwd_n = rec.rc_n = 0;
            rec.fwd_ref = rec.rc_ref = 0;
            rec.offset = 0;
            bool np = false;
            if (i < ng) {
                bool p0 = false;
                const int o = seed_offset(i, m, s, a.shifts, a.n_shifts, &p0);
                const uint64_t v = get32(a.rwords, rb + (uint64_t)o) & kmer_mask(s);
                uint32_t cnt = 0;
                lookup_seed(a.slots, a.T, a.positions, v, s, &rec, &cnt, a.status, &steps);
                rec.offset = (uint16_t)o;
                np = cnt <= (uint32_t)a.h_max;
            }
            unsigned hsum = np ? (unsigned)rec.fwd_n + rec.rc_n : 0u;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) hsum += __shfl_xor_sync(kFull, hsum, o);
            H += hsum;
            const unsigned npm = __ballot_sync(kFull, np);
            nnp += __popc(npm);
            for (unsigned mm = npm; mm && !full; mm &= mm - 1) {
                const int src = __ffs(mm) - 1;
                const uint32_t fref = __shfl_sync(kFull, rec.fwd_ref, src);
                const uint32_t rref = __shfl_sync(kFull, rec.rc_ref, src);
                const int fn = __shfl_sync(kFull, (int)rec.fwd_n, src);
                const int tot = fn + __shfl_sync(kFull, (int)rec.rc_n, src);
                const int o = __shfl_sync(kFull, (int)rec.offset, src);
                const int fl = __shfl_sync(kFull, (int)rec.flags, src);
                for (int j0 = 0; j0 < tot && !full; j0 += 32) {
                    const int j = j0 + lane;
                    bool ins = false;
                    if (j < tot) {
                        const bool fwd = j < fn;
                        const uint32_t l = fwd ? ((fl & kSeedFwdInline) ? fref
                                                                        : __ldg(a.positions + fref + j))
                                               : ((fl & kSeedRcInline) ? rref
                                                                       : __ldg(a.positions + rref + j - fn));
                        const long long p = fwd ? (long long)l - o : (long long)l - (m - o - s);
                        if (p >= 0) {
                            const unsigned long long key = 2ull * (unsigned long long)p + (fwd ? 0 : 1);
                            uint32_t h = (uint32_t)mix64(key) & (kCostSlots - 1);
                            for (int step = 0; step < kCostSlots; ++step) {
                                const unsigned long long prev = atomicCAS(&hs[h], kEmptyKey, key);
                                if (prev == kEmptyKey) ins = true;
                                if (prev == kEmptyKey || prev == key) break;
                                h = (h + 1) & (kCostSlots - 1);
                            }
                        }
                    }
                    nd += __popc(__ballot_sync(kFull, ins));
                    full = nd > kCostSlots / 2;  // so the set never holds more than 544 keys
                }
            }
        }
        if (lane == 0) {
            const int est = full ? nnp : min(nnp, nd);
            a.cost[r] = (uint32_t)min(est, kCostBuckets - 1);
            a.read_nd[r] = full ? kNoCount : (uint32_t)nd;
            atomicMax(a.need + q, full ? H : (unsigned)nd);
        }
        __syncwarp();
        for (int j = lane; j < kCostSlots; j += 32) hs[j] = kEmptyKey;
        __syncwarp();
    }
}

// One block of kScanThreads: out = the *count ids of `in` ordered by cost,
// largest first (ties in any order).
__global__ void __launch_bounds__(kScanThreads) k_order_by_cost(const uint32_t* in, uint32_t* out,
                                                                 const unsigned long long* count,
                                                                 const uint32_t* cost) {
    constexpr int kPer = kCostBuckets / kScanThreads;
    __shared__ uint32_t cur[kCostBuckets];
    __shared__ uint32_t wsum[kScanThreads / 32];
    const int tid = threadIdx.x;
    const unsigned long long n = *count;
    for (int b = tid; b < kCostBuckets; b += kScanThreads) cur[b] = 0;
    __syncthreads();
    // bucket kCostBuckets - 1 - cost: the scan then lays the largest costs out first
    for (unsigned long long it = tid; it < n; it += kScanThreads)
        atomicAdd(&cur[kCostBuckets - 1 - min(cost[in[it]], (uint32_t)(kCostBuckets - 1))], 1u);
    __syncthreads();
    uint32_t mine[kPer], sum = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        mine[k] = cur[tid * kPer + k];
        sum += mine[k];
    }
    uint32_t total;
    uint32_t start = block_exclusive_scan(sum, wsum, &total);
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        cur[tid * kPer + k] = start;
        start += mine[k];
    }
    __syncthreads();
    for (unsigned long long it = tid; it < n; it += kScanThreads) {
        const uint32_t id = in[it];
        const uint32_t b = kCostBuckets - 1 - min(cost[id], (uint32_t)(kCostBuckets - 1));
        out[atomicAdd(&cur[b], 1u)] = id;
    }
}

using FusedKernel = void (*)(FusedArgs);

// The kernel variant for a batch whose largest limit is Lmax: one or two
// register diagonals per lane when they cover [-Lmax, Lmax], else shared memory,
// with the q-gram bound when some read of the class can use it (qmaps).
static FusedKernel fused_kernel_for(int Lmax, bool qmaps, bool variant) {
    if (variant) {
        if (Lmax <= 15) return k_align_fused<1, true>;
        if (Lmax <= 31) return k_align_fused<2, true>;
        return qmaps ? k_align_fused<-1, true> : k_align_fused<0, true>;
    }
    if (Lmax <= 15) return k_align_fused<1, false>;
    if (Lmax <= 31) return k_align_fused<2, false>;
    return qmaps ? k_align_fused<-1, false> : k_align_fused<0, false>;
}

// The parameters that need the per-seed pick marks (see align_one_read).
static bool param_variant(const snap_index* idx, const snap_params* p) {
    return idx->stride > 1 || p->first_seeds > 1;
}

static bool is_team_kernel(FusedKernel k) {
    return k == k_align_team<false> || k == k_align_team<true> || k == k_align_wave;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int DevBuf::ensure(size_t need, const char* what) {
    if (need <= bytes && p) return SNAP_OK;
    std::lock_guard<std::recursive_mutex> lock(capture_alloc_mutex());
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    size_t want = std::max(need, (size_t)256);
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        set_error("out of device memory for %s (%zu bytes)", what, want);
        return SNAP_E_NOMEM;
    }
    bytes = want;
    return SNAP_OK;
}
void DevBuf::release() {
    std::lock_guard<std::recursive_mutex> lock(capture_alloc_mutex());
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
}
int PinnedBuf::ensure(size_t need, const char* what) {
    if (need <= bytes && p) return SNAP_OK;
    std::lock_guard<std::recursive_mutex> lock(capture_alloc_mutex());
    if (p) cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
    size_t want = std::max(need, (size_t)256);
    cudaError_t e = cudaMallocHost(&p, want);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        set_error("out of pinned host memory for %s", what);
        return SNAP_E_NOMEM;
    }
    bytes = want;
    return SNAP_OK;
}
void PinnedBuf::release() {
    std::lock_guard<std::recursive_mutex> lock(capture_alloc_mutex());
    if (p) cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
}



Engine* engine_create() {
    Engine* e = new Engine();
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&e->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e->sms <= 0) e->sms = 152;
    return e;
}

void engine_destroy(Engine* e) {
    if (!e) return;
    for (DevBuf& b : e->gseeds) b.release();
    for (DevBuf& b : e->gqbits) b.release();
    for (DevBuf* b : {&e->stats, &e->head, &e->packed, &e->gtab, &e->ghits, &e->gdense,
                      &e->heavy, &e->hseeds, &e->hprobed, &e->rcost, &e->rnd, &e->order2,
                      &e->cneed, &e->h_reads, &e->h_offsets, &e->h_out,
                      &e->h_dmax, &e->p_seeds,
                      &e->p_hits,
                      &e->p_hitoff, &e->p_partial, &e->p_table, &e->p_events, &e->p_hitlist,
                      &e->p_items, &e->p_misc, &e->p_dense})
        b->release();
    e->pin.release();
    for (auto& ev : e->ev)
        if (ev) cudaEventDestroy(ev);
    for (auto& ev : e->pev)
        if (ev) cudaEventDestroy(ev);
    for (auto& ev : e->tev)
        if (ev) cudaEventDestroy(ev);
    for (auto& ev : e->ev_join)
        if (ev) cudaEventDestroy(ev);
    if (e->ev_fork) cudaEventDestroy(e->ev_fork);
    for (auto& st : e->aux)
        if (st) cudaStreamDestroy(st);
    if (e->gexec) cudaGraphExecDestroy(e->gexec);
    if (e->own_stream) cudaStreamDestroy(e->own_stream);
    delete e;
}

size_t engine_bytes(const Engine* e) {
    size_t s = 0;
    for (const DevBuf& b : e->gseeds) s += b.bytes;
    for (const DevBuf& b : e->gqbits) s += b.bytes;
    for (const DevBuf* b : {&e->stats, &e->head, &e->packed, &e->gtab, &e->ghits, &e->gdense,
                            &e->heavy, &e->hseeds, &e->hprobed, &e->rcost, &e->rnd, &e->order2,
                            &e->cneed, &e->h_reads, &e->h_offsets, &e->h_out, &e->h_dmax,
                            &e->p_seeds,
                            &e->p_hits, &e->p_hitoff, &e->p_partial, &e->p_table, &e->p_events,
                            &e->p_hitlist, &e->p_items, &e->p_misc, &e->p_dense})
        s += b->bytes;
    return s;
}

void engine_release(Engine* e) {
    for (DevBuf& b : e->gseeds) b.release();
    for (DevBuf& b : e->gqbits) b.release();
    if (e->gexec) {
        cudaGraphExecDestroy(e->gexec);  // it points into the workspaces
        e->gexec = nullptr;
    }
    e->gtab_ready = false;
    for (DevBuf* b : {&e->packed, &e->gtab, &e->ghits, &e->gdense, &e->heavy, &e->hseeds,
                      &e->hprobed, &e->rcost, &e->rnd, &e->order2, &e->cneed, &e->h_reads,
                      &e->h_offsets,
                      &e->h_out, &e->h_dmax, &e->p_seeds, &e->p_hits, &e->p_hitoff, &e->p_partial,
                      &e->p_table, &e->p_events, &e->p_hitlist, &e->p_items, &e->p_misc, &e->p_dense})
        b->release();
}

void shift_list(int s, uint8_t* out, int* n_out) {
    // 0, then floor(j*s/2^k) for k = 1, 2, ... and odd j < 2^k, without repeats
    bool used[33] = {false};
    int n = 0;
    out[n++] = 0;
    used[0] = true;
    for (int k = 1; n < s && k < 40; ++k) {
        for (long long j = 1; j < (1ll << k) && n < s; j += 2) {
            const int d = (int)((j * s) >> k);
            if (!used[d]) {
                used[d] = true;
                out[n++] = (uint8_t)d;
            }
        }
    }
    *n_out = n;
}

int validate_params(const snap_index* idx, const snap_params* p) {
    if (!idx) {
        set_error("index is NULL");
        return SNAP_E_INVAL;
    }
    if (!p) {
        set_error("params is NULL");
        return SNAP_E_INVAL;
    }
    if (p->max_dist < 0) {
        set_error("max_dist %d < 0", p->max_dist);
        return SNAP_E_INVAL;
    }
    if (p->conf_diff < 1) {
        set_error("conf_diff %d < 1", p->conf_diff);
        return SNAP_E_INVAL;
    }
    if (p->max_hits < 0 || p->max_hits > (int)kListMax) {
        set_error("max_hits %d outside [0, %u]", p->max_hits, kListMax);
        return SNAP_E_INVAL;
    }
    if (p->collapse_duplicates != 0 && p->collapse_duplicates != 1) {
        set_error("collapse_duplicates %d is neither 0 nor 1", p->collapse_duplicates);
        return SNAP_E_INVAL;
    }
    if (p->first_seeds < 0 || p->first_seeds > kMaxSeeds) {
        set_error("first_seeds %d outside [0, %d]", p->first_seeds, kMaxSeeds);
        return SNAP_E_INVAL;
    }
    if (p->num_seeds < 0 || p->num_seeds > kMaxSeeds) {
        set_error("num_seeds %d outside [0, %d]", p->num_seeds, kMaxSeeds);
        return SNAP_E_INVAL;
    }
    return SNAP_OK;
}

int status_to_code(int st, const char* where) {
    if (!st) return SNAP_OK;
    if (st & kStBadBase) {
        set_error("%s: a read has a byte other than A, C, G, T", where);
        return SNAP_E_INVAL;
    }
    if (st & kStBadOffsets) {
        set_error("%s: read offsets decrease", where);
        return SNAP_E_INVAL;
    }
    if (st & kStReadTooLong) {
        set_error("%s: a read is longer than %d bases", where, kMaxReadLen);
        return SNAP_E_INVAL;
    }
    if (st & kStTooManySeeds) {
        set_error("%s: a read would use more than %d seeds", where, kMaxSeeds);
        return SNAP_E_INVAL;
    }
    if (st & kStBadDmax) {
        set_error("%s: a per-read max_dist is negative", where);
        return SNAP_E_INVAL;
    }
    if (st & kStTimeout) {
        set_error("%s: a bounded device wait gave up", where);
        return SNAP_E_TIMEOUT;
    }
    set_error("%s: device status 0x%x", where, st);
    return SNAP_E_INTERNAL;
}




int prepare_batch(const snap_index* idx, Engine* e, const uint8_t* d_reads,
                         const uint64_t* d_offsets, uint64_t n, const snap_params* p,
                         cudaStream_t stream, BatchPrep* out, const char* where) {
    int rc;
    if ((rc = e->stats.ensure(sizeof(BatchStats) + 64, "batch stats"))) return rc;
    if ((rc = e->pin.ensure(4096, "pinned stats"))) return rc;
    BatchStats* d_st = static_cast<BatchStats*>(e->stats.p);
    if (!e->ev[0])
        for (auto& ev : e->ev) SNAP_CUDA(cudaEventCreate(&ev), "event create");
    e->launches = 0;
    SNAP_CUDA(cudaEventRecord(e->ev[0], stream), "event");
    SNAP_CUDA(cudaMemsetAsync(d_st, 0, sizeof(BatchStats), stream), "stats clear");
    e->launches++;
    k_read_stats<<<stats_grid(e->sms, n), kStatsThreads, 0, stream>>>(
        d_offsets, n, idx->s, idx->stride, p->num_seeds, p->max_dist, p->conf_diff, p->max_hits,
        p->max_dist_per_read, d_st);
    SNAP_CUDA(cudaGetLastError(), "stats launch");
    BatchStats* h_st = static_cast<BatchStats*>(e->pin.p);
    uint64_t* h_base = reinterpret_cast<uint64_t*>(static_cast<char*>(e->pin.p) + 1024);
    SNAP_CUDA(cudaEventRecord(e->ev[1], stream), "event");
    SNAP_CUDA(cudaMemcpyAsync(h_st, d_st, sizeof(BatchStats), cudaMemcpyDeviceToHost, stream),
              "stats copy");
    SNAP_CUDA(cudaMemcpyAsync(h_base, d_offsets, sizeof(uint64_t), cudaMemcpyDeviceToHost, stream),
              "offset copy");
    SNAP_CUDA(cudaStreamSynchronize(stream), where);
    e->t_stats = std::chrono::steady_clock::now();
    out->st = *h_st;
    out->base0 = *h_base;
    if (out->st.status) return status_to_code(out->st.status, where);
    const uint64_t nwords = (out->st.total_bases + kReadPadBases + 15) / 16 + 8;
    if ((rc = e->packed.ensure(nwords * 4, "packed reads"))) return rc;
    out->rwords = static_cast<uint32_t*>(e->packed.p);
    const int aligned = ((reinterpret_cast<uintptr_t>(d_reads) + out->base0) % 16) == 0;
    int* d_status = &d_st->status;
    e->launches++;
    k_pack_reads<<<grid_cap(e->sms, nwords, 256), 256, 0, stream>>>(
        d_reads, out->base0, out->st.total_bases, out->rwords, nwords, aligned, d_status);
    SNAP_CUDA(cudaGetLastError(), "pack launch");
    SNAP_CUDA(cudaEventRecord(e->ev[2], stream), "event");
    return SNAP_OK;
}

// Milliseconds between two recorded events, 0 when the runtime cannot tell; a
// failure here is not left behind as the thread's last CUDA error.
static double event_ms(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return ms;
}

static int finish_status(Engine* e, cudaStream_t stream, const char* where, uint64_t n) {
    BatchStats* d_st = static_cast<BatchStats*>(e->stats.p);
    SNAP_CUDA(cudaEventRecord(e->ev[3], stream), "event");
    BatchStats* h = reinterpret_cast<BatchStats*>(static_cast<char*>(e->pin.p) + 2048);
    SNAP_CUDA(cudaMemcpyAsync(h, d_st, sizeof(BatchStats), cudaMemcpyDeviceToHost, stream),
              "status copy");
    SNAP_CUDA(cudaStreamSynchronize(stream), where);
    const int rc = status_to_code(h->status, where);
    if (rc) return rc;
    snap_call_stats& L = e->last;
    L.kernel_launches = e->launches;
    L.stats_ms = event_ms(e->ev[0], e->ev[1]);
    L.pack_ms = event_ms(e->ev[1], e->ev[2]);
    L.align_ms = event_ms(e->ev[2], e->ev[3]);
    L.total_ms = event_ms(e->ev[0], e->ev[3]);
    L.reads = n;
    L.read_bases = h->total_bases;
    L.seeds = h->ctr.seeds;
    L.slot_reads = h->ctr.slot_reads;
    L.list_entries = h->ctr.list_entries;
    L.ed_calls = h->ctr.ed_calls;
    L.ed_over = h->ctr.ed_over;
    L.window_bytes = h->ctr.window_words * 4;
    L.ed_filtered = h->ctr.ed_filtered;
    L.ed_collapsed = h->ctr.ed_collapsed;
    L.light_threads = e->last_shape.light_threads;
    L.warps_per_block = e->last_shape.warps;
    L.table_slots = e->last_shape.scap;
    L.graph_replay = e->last_graph;
    L.team_classes = e->last_team;
    L.wave_classes = e->last_wave;
    L.wave_warps = e->last_wave_warps;
    L.probe_ms = L.distance_ms = 0;
    L.host_plan_ms = e->host_plan_ms;
    L.reads_light = h->ctr_light.reads_done;
    L.light_seeds = h->ctr_light.seeds;
    L.light_slot_reads = h->ctr_light.slot_reads;
    L.light_list_entries = h->ctr_light.list_entries;
    L.light_ed_calls = h->ctr_light.ed_calls;
    L.light_window_bytes = h->ctr_light.window_words * 4;
    L.light_ms = 0;
    if (e->last_light && h->light_end_ns > ~h->light_start_ns_neg)
        L.light_ms = (double)(h->light_end_ns - ~h->light_start_ns_neg) * 1e-6;
    if (e->last_plain) {
        L.probe_ms = event_ms(e->pev[3], e->pev[0]);
        L.distance_ms = event_ms(e->pev[1], e->pev[2]);
    }
    return SNAP_OK;
}

// The launch plan of the batched form for one shape: whether the thread-per-read
// kernel runs, and one warp-kernel launch per non-empty read-length class, each
// laid out for its class's longest read and largest limit.
struct BatchPlan {
    LaunchShape shape;
    bool light = false;
    bool use[kClasses] = {false, false, false, false};
    FusedArgs a[kClasses];
    FusedKernel kfn[kClasses] = {nullptr, nullptr, nullptr, nullptr};
    size_t smem[kClasses] = {0, 0, 0, 0};
    uint64_t blocks[kClasses] = {0, 0, 0, 0};
    int warps[kClasses] = {0, 0, 0, 0};    // reads in flight per block
    int threads[kClasses] = {0, 0, 0, 0};  // threads per block
    ClassLists cl;
    uint32_t* heavy_ids = nullptr;
    unsigned long long* head = nullptr;  // [0..3] class queue heads, [4] leftovers, [5..8] class counts
    uint64_t table_slots[kClasses] = {0, 0, 0, 0};  // global candidate slots each class needs
    bool ordered[kClasses] = {false, false, false, false};  // k_order_by_cost before the launch
    bool counted[kClasses] = {false, false, false, false};  // per-read table bounds (read_nd)
    const uint32_t* unsorted[kClasses] = {nullptr, nullptr, nullptr, nullptr};
    uint32_t* rcost = nullptr;
    uint32_t* rnd = nullptr;
    bool concurrent = false;  // class launches side by side (disjoint global tables)
};

// Whether class q aligns one read per block (team or wave mode): its limits
// exceed 31 and (chosen per batch) it has fewer than max(8, longest read / 12)
// reads per SM, where per-read work, growing with the square of the limit, would
// leave one warp per read latency-bound; e->team: -1 per batch, 0 never, >= 1 always.
static bool block_per_read(const Engine* e, const BatchPrep& bp, int q) {
    const int mmax = std::max(1u, bp.st.cls_max_len[q]);
    const int Lmax = std::max(0, bp.st.cls_max_L0[q]);
    const uint64_t team_below = (uint64_t)e->sms * std::max(kTeamReadsPerSm, mmax / 12);
    return Lmax > 31 && (e->team < 0 ? bp.st.cls_n[q] < team_below : e->team >= 1);
}

// k_read_cost over the reads of the block-per-read classes (plain index,
// first_seeds <= 1): per-read cost keys and distinct-candidate counts on the
// device, each class's largest table need on the host (e->cost_need).
static int count_candidates(const snap_index* idx, Engine* e, const uint64_t* d_offsets,
                            uint64_t n, const snap_params* p, cudaStream_t stream,
                            const BatchPrep& bp) {
    int rc;
    e->cost_mask = e->len_mask = 0;
    if (param_variant(idx, p)) return SNAP_OK;
    for (int q = 0; q < kClasses; ++q) {
        if (!bp.st.cls_n[q]) continue;
        if (block_per_read(e, bp, q))
            e->cost_mask |= 1u << q;
        else if (bp.st.cls_max_L0[q] > 31)
            e->len_mask |= 1u << q;  // warp per read, costs spread with the square of m
    }
    if (!e->cost_mask && !e->len_mask) return SNAP_OK;
    if ((rc = e->rcost.ensure(n * sizeof(uint32_t), "read costs"))) return rc;
    if ((rc = e->rnd.ensure(n * sizeof(uint32_t), "candidate counts"))) return rc;
    if ((rc = e->cneed.ensure(kClasses * sizeof(unsigned), "table needs"))) return rc;
    SNAP_CUDA(cudaMemsetAsync(e->cneed.p, 0, kClasses * sizeof(unsigned), stream), "need clear");
    CostArgs ca;
    memset(&ca, 0, sizeof(ca));
    ca.offsets = d_offsets;
    ca.n = n;
    ca.rwords = bp.rwords;
    ca.base0 = bp.base0;
    ca.s = idx->s;
    ca.num_seeds = p->num_seeds;
    ca.h_max = p->max_hits;
    shift_list(idx->s, ca.shifts, &ca.n_shifts);
    ca.slots = idx->slots;
    ca.T = idx->T;
    ca.positions = idx->positions;
    ca.status = &static_cast<BatchStats*>(e->stats.p)->status;
    ca.mask = e->cost_mask;
    ca.len_mask = e->len_mask;
    ca.cost = static_cast<uint32_t*>(e->rcost.p);
    ca.read_nd = static_cast<uint32_t*>(e->rnd.p);
    ca.need = static_cast<unsigned*>(e->cneed.p);
    const unsigned blocks = (unsigned)std::max<uint64_t>(
        1, std::min<uint64_t>((uint64_t)e->sms * 16, (n + kCostWarps - 1) / kCostWarps));
    e->launches++;
    k_read_cost<<<blocks, kCostWarps * 32, 0, stream>>>(ca);
    SNAP_CUDA(cudaGetLastError(), "cost launch");
    if (!e->cost_mask) return SNAP_OK;  // length keys only: nothing to read back
    unsigned* h_need = reinterpret_cast<unsigned*>(static_cast<char*>(e->pin.p) + 3200);
    SNAP_CUDA(cudaMemcpyAsync(h_need, e->cneed.p, kClasses * sizeof(unsigned),
                              cudaMemcpyDeviceToHost, stream), "need copy");
    SNAP_CUDA(cudaStreamSynchronize(stream), "snap_align");
    for (int q = 0; q < kClasses; ++q) e->cost_need[q] = h_need[q];
    return SNAP_OK;
}

// Lay out the warp kernel of class q; allocate what it needs (no allocation
// happens after planning, so the enqueue can be captured).
static int plan_class(const snap_index* idx, Engine* e, const uint64_t* d_offsets, uint64_t n,
                      const snap_params* p, snap_result* d_out, const BatchPrep& bp,
                      const LaunchShape& shape, int q, cudaStream_t stream, BatchPlan* plan) {
    int rc;
    FusedArgs& a = plan->a[q];
    memset(&a, 0, sizeof(a));
    a.genome = idx->genome_words;
    a.G = idx->G;
    a.s = idx->s;
    a.slots = idx->slots;
    a.T = idx->T;
    a.positions = idx->positions;
    a.rwords = bp.rwords;
    a.offsets = d_offsets;
    a.base0 = bp.base0;
    a.order = plan->cl.list + plan->cl.off[q];
    a.n_items = n;
    a.n_items_dev = plan->cl.count + q;
    a.head = plan->head + q;
    a.d_max = p->max_dist;
    a.h_max = p->max_hits;
    a.c = p->conf_diff;
    a.num_seeds = p->num_seeds;
    a.first_seeds = p->first_seeds;
    a.collapse = p->collapse_duplicates;
    a.stride = idx->stride;
    a.dmax_per_read = p->max_dist_per_read;
    shift_list(idx->s, a.shifts, &a.n_shifts);
    a.out = d_out;
    a.status = &static_cast<BatchStats*>(e->stats.p)->status;
    a.ctr = &static_cast<BatchStats*>(e->stats.p)->ctr;
    const int mmax = std::max(1u, bp.st.cls_max_len[q]);
    const int Lmax = std::max(0, bp.st.cls_max_L0[q]);
    const int nmax = std::max(1, bp.st.cls_max_seeds[q]);
    auto up4 = [](int w) { return (w + 3) & ~3; };
    a.wx = up4((mmax + 15) / 16 + 4);
    a.wt = up4((mmax + Lmax + 15 + 15) / 16 + 4);
    a.seed_cap = nmax;
    a.lv_ints = Lmax > 31 ? up4(2 * (2 * Lmax + 4)) : 0;
    // many seeds (long reads): seed records in global memory, more warps per SM
    const bool seeds_global = nmax > 64;
    const int seed_words = seeds_global ? 0 : 4 * a.seed_cap;
    const bool team = block_per_read(e, bp, q);
    const bool ordered = (e->cost_mask >> q) & 1u;  // counted by k_read_cost
    const bool by_length = (e->len_mask >> q) & 1u;  // keyed by read length
    const int pwords = (Lmax <= 31 && !team) ? par_words(mmax) : 0;  // register-diagonal kernels
    const int fixed_words = 2 * a.wx + a.wt + seed_words + a.lv_ints + pwords;
    const int budget_words = 200 * 1024 / 4;  // per block; 7 words per table slot
    // a class of large limits with too few reads to give each SM several warps
    // runs in team mode (a block per read, `team` above); `warps` counts the
    // per-read warps (lead warps) of a block, which own the per-warp layout below
    int warps = team ? 1 : std::max(1, shape.warps);
    // a class with few reads spreads them over all SMs (one warp per read)
    while (warps > 1 && bp.st.cls_n[q] < (uint64_t)e->sms * warps) warps >>= 1;
    while (warps > 1 && warps * (fixed_words + 7 * 64) > budget_words) warps >>= 1;
    int scap = std::max(64, shape.scap);
    if (ordered) {
        // room in shared memory for the largest distinct-candidate count of the
        // class, up to 1024 slots (one table per block in this mode)
        uint32_t want = 64;
        while (want < 2u * std::min(e->cost_need[q], 512u)) want <<= 1;
        scap = std::max(scap, (int)want);
    }
    while (scap > 64 && warps * (fixed_words + 7 * scap) > budget_words) scap >>= 1;
    a.scap = scap;
    a.off_xr = a.wx;
    a.off_tw = 2 * a.wx;
    a.off_seeds = a.off_tw + a.wt;
    a.off_tab = a.off_seeds + seed_words;         // SeedRec: 4 words
    a.off_hits = a.off_tab + 4 * scap;            // CandSlot: 4 words
    a.off_dense = a.off_hits + 4 * (scap / 2);    // HitRec: 4 words, scap/2 of them
    a.off_lv = a.off_dense + up4(scap / 2);       // dense slot list: scap/2 words
    a.off_par = pwords ? a.off_lv + a.lv_ints : 0;
    a.par_mmax = mmax;
    a.warp_words = a.off_lv + a.lv_ints + pwords;
    if ((a.off_seeds | a.off_tab | a.off_hits | a.off_dense | a.off_lv | a.off_par |
         a.warp_words) & 3) {
        set_error("snap_align: internal shared-memory layout is not 16-byte aligned");
        return SNAP_E_INTERNAL;
    }
    size_t smem = (size_t)warps * a.warp_words * 4 + (team ? kJobWords * 4 : 0);
    const bool variant = param_variant(idx, p);
    // wave mode (asked for with team = 2): the number of warps (candidates per
    // wave) that puts the most warps on an SM, at most kWaveMaxWarps, ties to
    // more per block
    int wave_warps = 0;
    if (team && !variant && e->team == 2) {
        int best = 0;
        for (int W = kWaveMaxWarps; W >= 2; W >>= 1) {
            const size_t b = ((size_t)a.warp_words + (size_t)(W - 1) * (a.wt + a.lv_ints) +
                              kWaveJobWords) * 4;
            if (b > 227 * 1024) continue;
            if ((rc = raise_smem_limit((const void*)k_align_wave, b))) return rc;
            int per_sm = 0;
            SNAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_align_wave, W * 32, b),
                      "occupancy");
            if (per_sm * W > best) {
                best = per_sm * W;
                wave_warps = W;
            }
        }
        if (wave_warps)
            smem = ((size_t)a.warp_words + (size_t)(wave_warps - 1) * (a.wt + a.lv_ints) +
                    kWaveJobWords) * 4;
    }
    if (smem > 227 * 1024) {
        set_error("snap_align: read length %d needs %zu bytes of shared memory per warp", mmax,
                  (size_t)a.warp_words * 4);
        return SNAP_E_INVAL;
    }
    // q-gram maps only when some read of the class can use the bound: for limit
    // L the read length must lie in [9L - 7, L^2 / 8 - L]
    bool qmaps = false;
    for (int L = kQMinL; L <= Lmax && !qmaps; ++L)
        qmaps = use_qfilter(std::min(mmax, L * L / 8 - L), L);
    const FusedKernel kfn = wave_warps ? k_align_wave
                            : team     ? (variant ? k_align_team<true> : k_align_team<false>)
                                       : fused_kernel_for(Lmax, qmaps, variant);
    const int threads = wave_warps ? wave_warps * 32 : team ? kTeamWarps * 32 : warps * 32;
    if ((rc = raise_smem_limit((const void*)kfn, smem))) return rc;
    int per_sm = 0;
    SNAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, threads, smem),
              "occupancy");
    if (per_sm < 1) per_sm = 1;
    uint64_t blocks = (uint64_t)e->sms * per_sm;
    const uint64_t need_blocks = (bp.st.cls_n[q] + warps - 1) / warps;
    if (blocks > need_blocks) blocks = std::max<uint64_t>(1, need_blocks);
    // global overflow tables for reads whose candidate table outgrows shared memory
    // (sized for the class's largest hit count, or its largest distinct count when
    // k_read_cost counted it)
    const uint64_t hb = ordered ? (uint64_t)e->cost_need[q] : bp.st.cls_max_hits[q];
    uint64_t gcap = 64;
    while (gcap < 2 * hb) gcap <<= 1;
    if (gcap > kMaxTableSlots) {
        set_error("snap_align: seeds x max_hits per read (%llu) exceeds %u",
                  (unsigned long long)hb, kMaxTableSlots / 2);
        return SNAP_E_INVAL;
    }
    if (gcap > (uint64_t)scap) {
        // the tables themselves are allocated in plan_batch once every class is laid out
        const uint64_t per_warp = gcap * (sizeof(CandSlot) + sizeof(HitRec) / 2 + 2);
        const uint64_t max_warps = std::max<uint64_t>(1, e->overflow_budget / per_warp);
        if (blocks * warps > max_warps) blocks = std::max<uint64_t>(1, max_warps / warps);
        a.gcap = (uint32_t)gcap;
        plan->table_slots[q] = blocks * warps * gcap;
    }
    if (qmaps) {
        // presence maps start zero; kernels clear what they set before the next read
        DevBuf& gq = e->gqbits[q];
        void* before = gq.p;
        const size_t before_bytes = gq.bytes;
        if ((rc = gq.ensure(blocks * warps * 2ull * kQWords * sizeof(uint32_t), "q-gram maps")))
            return rc;
        if (gq.p != before || gq.bytes != before_bytes)
            SNAP_CUDA(cudaMemsetAsync(gq.p, 0, gq.bytes, stream), "q-gram map init");
        a.gqbits = static_cast<uint32_t*>(gq.p);
    }
    if (seeds_global) {
        DevBuf& gs = e->gseeds[q];
        if ((rc = gs.ensure(blocks * warps * (uint64_t)a.seed_cap * sizeof(SeedRec),
                            "seed records")))
            return rc;
        a.gseeds = static_cast<SeedRec*>(gs.p);
    }
    // a block-per-read class runs its reads largest estimate first (k_read_cost),
    // a warp-per-read class of large limits its longest reads first
    plan->ordered[q] = ordered || by_length;
    plan->counted[q] = ordered;
    plan->kfn[q] = kfn;
    plan->smem[q] = smem;
    plan->blocks[q] = blocks;
    plan->warps[q] = warps;
    plan->threads[q] = threads;
    plan->use[q] = true;
    return SNAP_OK;
}

static int plan_batch(const snap_index* idx, Engine* e, const uint64_t* d_offsets, uint64_t n,
                      const snap_params* p, snap_result* d_out, const BatchPrep& bp,
                      const LaunchShape& shape, cudaStream_t stream, BatchPlan* plan) {
    int rc;
    plan->shape = shape;
    plan->light = bp.st.n_light > 0 && shape.light_threads > 0;
    if ((rc = e->head.ensure(16 * sizeof(unsigned long long), "queue heads"))) return rc;
    plan->head = static_cast<unsigned long long*>(e->head.p);
    if ((rc = e->heavy.ensure(2 * n * sizeof(uint32_t), "read lists"))) return rc;
    plan->heavy_ids = static_cast<uint32_t*>(e->heavy.p);
    plan->cl.list = plan->heavy_ids + n;
    plan->cl.count = plan->head + 5;
    unsigned long long off = 0;
    for (int q = 0; q < kClasses; ++q) {
        plan->cl.off[q] = off;
        off += bp.st.cls_n[q];
    }
    if (plan->light) {
        if ((rc = light_prepare())) return rc;
        if ((rc = e->hseeds.ensure(n * kLightHandoverSlots * sizeof(SeedRec), "handed-over probes")))
            return rc;
        if ((rc = e->hprobed.ensure(n, "handed-over flags"))) return rc;
    }
    for (int q = 0; q < kClasses; ++q)
        if (bp.st.cls_n[q] > 0 &&
            (rc = plan_class(idx, e, d_offsets, n, p, d_out, bp, shape, q, stream, plan)))
            return rc;
    for (int q = 0; q < kClasses; ++q) {
        plan->a[q].hseeds = plan->light ? static_cast<const SeedRec*>(e->hseeds.p) : nullptr;
        plan->a[q].hprobed = plan->light ? static_cast<const uint8_t*>(e->hprobed.p) : nullptr;
    }
    bool any_ordered = false;
    for (int q = 0; q < kClasses; ++q) any_ordered |= plan->use[q] && plan->ordered[q];
    if (any_ordered) {
        if ((rc = e->rcost.ensure(n * sizeof(uint32_t), "read costs"))) return rc;
        if ((rc = e->rnd.ensure(n * sizeof(uint32_t), "candidate counts"))) return rc;
        if ((rc = e->order2.ensure(n * sizeof(uint32_t), "ordered read lists"))) return rc;
        plan->rcost = static_cast<uint32_t*>(e->rcost.p);
        plan->rnd = static_cast<uint32_t*>(e->rnd.p);
        for (int q = 0; q < kClasses; ++q) {
            if (!plan->use[q] || !plan->ordered[q]) continue;
            plan->unsorted[q] = plan->cl.list + plan->cl.off[q];
            plan->a[q].order = static_cast<uint32_t*>(e->order2.p) + plan->cl.off[q];
            plan->a[q].read_nd = plan->counted[q] ? plan->rnd : nullptr;
        }
    }
    // global candidate tables: the class launches run side by side when two or
    // more classes are present and their tables fit the budget together (each
    // class its own slice), else one after another sharing one buffer for the
    // largest need; kernels leave their tables empty
    const uint64_t slot_bytes = sizeof(CandSlot) + sizeof(HitRec) / 2 + sizeof(uint32_t) / 2;
    int nuse = 0, ntab = 0;
    uint64_t slots_sum = 0, slots_max = 0;
    for (int q = 0; q < kClasses; ++q) {
        nuse += plan->use[q];
        ntab += plan->table_slots[q] > 0;
        slots_sum += plan->table_slots[q];
        slots_max = std::max(slots_max, plan->table_slots[q]);
    }
    plan->concurrent = nuse >= 2 && (ntab <= 1 || slots_sum * slot_bytes <= e->overflow_budget);
    const uint64_t slots = plan->concurrent ? slots_sum : slots_max;
    if (slots) {
        void* before = e->gtab.p;
        const size_t before_bytes = e->gtab.bytes;
        if ((rc = e->gtab.ensure(slots * sizeof(CandSlot), "overflow tables"))) return rc;
        if ((rc = e->ghits.ensure(slots / 2 * sizeof(HitRec), "overflow hits"))) return rc;
        if ((rc = e->gdense.ensure(slots / 2 * sizeof(uint32_t), "overflow lists"))) return rc;
        if (e->gtab.p != before || e->gtab.bytes != before_bytes || !e->gtab_ready) {
            // fresh tables start empty; kernels keep them empty afterwards
            const uint64_t all = e->gtab.bytes / sizeof(CandSlot);
            k_init_ctab<<<grid_cap(e->sms, all, 256), 256, 0, stream>>>(
                static_cast<CandSlot*>(e->gtab.p), all);
            SNAP_CUDA(cudaGetLastError(), "table init");
            e->gtab_ready = true;
        }
        uint64_t at = 0;  // this class's first slot
        for (int q = 0; q < kClasses; ++q) {
            if (!plan->table_slots[q]) continue;
            plan->a[q].gtab = static_cast<CandSlot*>(e->gtab.p) + at;
            plan->a[q].ghits = static_cast<HitRec*>(e->ghits.p) + at / 2;
            plan->a[q].gdense = static_cast<uint32_t*>(e->gdense.p) + at / 2;
            if (plan->concurrent) at += plan->table_slots[q];
        }
    }
    return SNAP_OK;
}

// Enqueue the planned launch sequence on `stream` (allocation-free; capturable).
static int enqueue_batch(const snap_index* idx, Engine* e, const uint64_t* d_offsets, uint64_t n,
                         const snap_params* p, snap_result* d_out, cudaStream_t stream,
                         const BatchPrep& bp, const BatchPlan& plan) {
    int rc;
    SNAP_CUDA(cudaMemsetAsync(plan.head, 0, 16 * sizeof(unsigned long long), stream),
              "queue clear");
    if (plan.light) {
        // short reads: one thread each; the leftovers go to the warp kernel
        SNAP_CUDA(cudaMemsetAsync(e->hprobed.p, 0, n, stream), "hand-over clear");
        if ((rc = launch_light(idx, e, d_offsets, n, p, d_out, stream, bp, plan.heavy_ids,
                               plan.head + 4, plan.shape.light_threads,
                               static_cast<SeedRec*>(e->hseeds.p),
                               static_cast<uint8_t*>(e->hprobed.p))))
            return rc;
    }
    e->launches++;
    k_split_classes<<<grid_cap(e->sms, n, 256), 256, 0, stream>>>(
        plan.light ? plan.heavy_ids : nullptr, plan.head + 4, n, d_offsets, plan.cl);
    SNAP_CUDA(cudaGetLastError(), "split launch");
    // the class launches, longest reads first; side by side, the first on the
    // caller's stream and each other one on its own stream forked from it
    if (plan.concurrent) {
        if (!e->ev_fork) {
            SNAP_CUDA(cudaEventCreateWithFlags(&e->ev_fork, cudaEventDisableTiming), "event create");
            for (int q = 0; q < kClasses; ++q) {
                SNAP_CUDA(cudaEventCreateWithFlags(&e->ev_join[q], cudaEventDisableTiming),
                          "event create");
                SNAP_CUDA(cudaStreamCreateWithFlags(&e->aux[q], cudaStreamNonBlocking),
                          "stream create");
            }
        }
        SNAP_CUDA(cudaEventRecord(e->ev_fork, stream), "fork");
    }
    bool forked[kClasses] = {false, false, false, false};
    bool first = true;
    for (int q = kClasses - 1; q >= 0; --q) {
        if (!plan.use[q]) continue;
        cudaStream_t sq = stream;
        if (plan.concurrent && !first) {
            sq = e->aux[q];
            SNAP_CUDA(cudaStreamWaitEvent(sq, e->ev_fork, 0), "fork");
            forked[q] = true;
        }
        first = false;
        if (plan.ordered[q]) {
            e->launches++;
            k_order_by_cost<<<1, kScanThreads, 0, sq>>>(plan.unsorted[q],
                                                        const_cast<uint32_t*>(plan.a[q].order),
                                                        plan.cl.count + q, plan.rcost);
            SNAP_CUDA(cudaGetLastError(), "order launch");
        }
        e->launches++;
        plan.kfn[q]<<<(unsigned)plan.blocks[q], plan.threads[q], plan.smem[q], sq>>>(plan.a[q]);
        SNAP_CUDA(cudaGetLastError(), "align launch");
        if (forked[q]) SNAP_CUDA(cudaEventRecord(e->ev_join[q], sq), "join");
    }
    for (int q = 0; q < kClasses; ++q)
        if (forked[q]) SNAP_CUDA(cudaStreamWaitEvent(stream, e->ev_join[q], 0), "join");
    return SNAP_OK;
}

// Launch shapes the tuner tries: threads per block of the thread-per-read
// bucket, warps per block and shared candidate slots of the warp kernel.
static const LaunchShape kShapes[] = {
    {128, 8, 128}, {64, 8, 128}, {256, 8, 128}, {128, 8, 64}, {128, 4, 256}, {128, 4, 128},
};

static bool same_key(const TuneKey& x, const TuneKey& y) {
    return x.lvd == y.lvd && x.light == y.light && x.mmax == y.mmax && x.Lmax == y.Lmax &&
           x.nmax == y.nmax && x.hits == y.hits && x.nbucket == y.nbucket;
}

static int align_fused(const snap_index* idx, Engine* e, const uint64_t* d_offsets, uint64_t n,
                       const snap_params* p, snap_result* d_out, cudaStream_t stream,
                       const BatchPrep& bp) {
    int rc;
    if ((rc = count_candidates(idx, e, d_offsets, n, p, stream, bp))) return rc;
    // batches that share the classes present, the limits' register layout, the
    // thread-per-read kernel and the size within a factor of two share a tuned shape
    TuneKey key;
    key.lvd = 0;
    for (int q = 0; q < kClasses; ++q)
        if (bp.st.cls_n[q]) key.lvd |= 1 << q;
    key.light = bp.st.n_light > 0;
    const int L = bp.st.max_L0;
    key.mmax = 0;
    key.Lmax = L <= 15 ? 15 : L <= 31 ? 31 : L <= 63 ? 63 : L <= 127 ? 127 : 1000;
    key.nmax = 0;
    key.hits = 0;
    int lg = 0;
    while ((1ull << lg) < n) ++lg;
    key.nbucket = lg;
    LaunchShape shape = kShapes[0];
    bool tuned = false;
    for (const auto& t : e->tuned)
        if (same_key(t.first, key)) {
            shape = t.second;
            tuned = true;
        }
    if (!tuned && e->autotune && n >= 4096) {
        // time candidate shapes on this batch (results do not depend on the
        // shape); give up on the search when one run is too slow to repeat
        if (!e->tev[0])
            for (auto& ev : e->tev) SNAP_CUDA(cudaEventCreate(&ev), "event create");
        float best_ms = 1e30f;
        for (const LaunchShape& cand : kShapes) {
            if (!key.light && cand.light_threads != kShapes[0].light_threads) continue;
            BatchPlan tp;
            if ((rc = plan_batch(idx, e, d_offsets, n, p, d_out, bp, cand, stream, &tp))) return rc;
            SNAP_CUDA(cudaEventRecord(e->tev[0], stream), "event");
            if ((rc = enqueue_batch(idx, e, d_offsets, n, p, d_out, stream, bp, tp))) return rc;
            SNAP_CUDA(cudaEventRecord(e->tev[1], stream), "event");
            SNAP_CUDA(cudaEventSynchronize(e->tev[1]), "tune");
            float ms = 0;
            SNAP_CUDA(cudaEventElapsedTime(&ms, e->tev[0], e->tev[1]), "tune");
            if (ms < best_ms) {
                best_ms = ms;
                shape = cand;
            }
            if (ms > 50.0f) break;
        }
        e->tuned.push_back({key, shape});
    }
    BatchPlan plan;
    if ((rc = plan_batch(idx, e, d_offsets, n, p, d_out, bp, shape, stream, &plan))) return rc;
    e->last_shape = shape;
    for (int q = 0; q < kClasses; ++q)
        if (plan.use[q]) {
            e->last_shape.warps = plan.threads[q] / 32;
            e->last_shape.scap = plan.a[q].scap;
            break;
        }
    e->last_team = e->last_wave = e->last_wave_warps = 0;
    for (int q = 0; q < kClasses; ++q) {
        e->last_team += plan.use[q] && is_team_kernel(plan.kfn[q]);
        if (plan.use[q] && plan.kfn[q] == k_align_wave) {
            e->last_wave++;
            e->last_wave_warps = plan.threads[q] / 32;
        }
    }
    e->last_light = plan.light;
    e->last_graph = 0;
    if (e->use_graphs && stream != nullptr && stream != cudaStreamLegacy &&
        stream != cudaStreamPerThread) {
        // capture the launch sequence and replay it as one graph; an existing
        // executable graph is updated in place when only parameters changed
        cudaGraph_t g = nullptr;
        cudaError_t ce;
        {
            std::lock_guard<std::recursive_mutex> lock(capture_alloc_mutex());
            SNAP_CUDA(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal), "capture");
            rc = enqueue_batch(idx, e, d_offsets, n, p, d_out, stream, bp, plan);
            ce = cudaStreamEndCapture(stream, &g);
        }
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        SNAP_CUDA(ce, "end capture");
        bool ok = false;
        if (e->gexec) {
            cudaGraphExecUpdateResultInfo info;
            ok = cudaGraphExecUpdate(e->gexec, g, &info) == cudaSuccess;
            if (!ok) {
                cudaGetLastError();
                cudaGraphExecDestroy(e->gexec);
                e->gexec = nullptr;
            }
        }
        if (!ok) {
            const cudaError_t ie = cudaGraphInstantiate(&e->gexec, g, 0);
            if (ie != cudaSuccess) {
                cudaGraphDestroy(g);
                e->gexec = nullptr;
                return cuda_fail(ie, "graph instantiate");
            }
        }
        cudaGraphDestroy(g);
        SNAP_CUDA(cudaGraphLaunch(e->gexec, stream), "graph launch");
        e->last_graph = 1;
    } else {
        if ((rc = enqueue_batch(idx, e, d_offsets, n, p, d_out, stream, bp, plan))) return rc;
    }
    return SNAP_OK;
}

int align_plain(const snap_index* idx, Engine* e, const uint64_t* d_offsets, uint64_t n,
                const snap_params* p, snap_result* d_out, cudaStream_t stream,
                const BatchPrep& bp);

int align_batch_device(const snap_index* idx, Engine* e, const uint8_t* d_reads,
                       const uint64_t* d_offsets, uint64_t n, const snap_params* p,
                       snap_result* d_out, cudaStream_t stream, bool plain) {
    int rc = validate_params(idx, p);
    if (rc) return rc;
    if (n == 0) return SNAP_OK;
    if (!d_reads || !d_offsets || !d_out) {
        set_error("snap_align: NULL buffer");
        return SNAP_E_INVAL;
    }
    if ((reinterpret_cast<uintptr_t>(d_offsets) | reinterpret_cast<uintptr_t>(d_out)) % 8 ||
        (p->max_dist_per_read && reinterpret_cast<uintptr_t>(p->max_dist_per_read) % 4)) {
        set_error("snap_align: offsets and results must be 8-byte aligned, max_dist_per_read "
                  "4-byte aligned");
        return SNAP_E_INVAL;
    }
    const char* where = plain ? "snap_align_plain" : "snap_align";
    e->last_shape = LaunchShape{0, 0, 0};  // set again by the batched form
    e->last_graph = 0;
    e->last_team = e->last_wave = e->last_wave_warps = 0;
    e->cost_mask = e->len_mask = 0;  // set by count_candidates for the batched form
    e->last_light = false;
    e->last_plain = plain;
    BatchPrep bp;
    if ((rc = prepare_batch(idx, e, d_reads, d_offsets, n, p, stream, &bp, where))) return rc;
    rc = plain ? align_plain(idx, e, d_offsets, n, p, d_out, stream, bp)
               : align_fused(idx, e, d_offsets, n, p, d_out, stream, bp);
    if (rc) return rc;
    e->host_plan_ms = std::chrono::duration<double, std::milli>(
                          std::chrono::steady_clock::now() - e->t_stats).count();
    return finish_status(e, stream, where, n);
}

// Host buffers: copy in, run the device path, copy out (engine-owned stream).
static int align_host(const snap_index* idx, const uint8_t* reads, const uint64_t* offsets,
                      uint64_t n, const snap_params* p, snap_result* out, bool plain) {
    clear_error();
    int rc = validate_params(idx, p);
    if (rc) return rc;
    if (n == 0) return SNAP_OK;
    if (!reads || !offsets || !out) {
        set_error("snap_align: NULL buffer");
        return SNAP_E_INVAL;
    }
    Engine* e = idx->engine;
    std::lock_guard<std::mutex> lock(e->mu);
    if (!e->own_stream) SNAP_CUDA(cudaStreamCreateWithFlags(&e->own_stream, cudaStreamNonBlocking),
                                  "stream create");
    cudaStream_t st = e->own_stream;
    const uint64_t lo = offsets[0], hi = offsets[n];
    if (hi < lo) {
        set_error("snap_align: read offsets decrease");
        return SNAP_E_INVAL;
    }
    const uint64_t bytes = hi - lo;
    if ((rc = e->h_reads.ensure(bytes + 16, "read copy"))) return rc;
    if ((rc = e->h_offsets.ensure((n + 1) * 8, "offset copy"))) return rc;
    if ((rc = e->h_out.ensure(n * sizeof(snap_result), "result buffer"))) return rc;
    SNAP_CUDA(cudaMemcpyAsync(e->h_reads.p, reads + lo, bytes, cudaMemcpyHostToDevice, st),
              "reads H2D");
    // offsets are rebased by the device path through base0; copy as given and
    // point the device reads at the copy's start minus lo
    SNAP_CUDA(cudaMemcpyAsync(e->h_offsets.p, offsets, (n + 1) * 8, cudaMemcpyHostToDevice, st),
              "offsets H2D");
    snap_params dp = *p;
    if (p->max_dist_per_read) {
        if ((rc = e->h_dmax.ensure(n * 4, "max_dist copy"))) return rc;
        SNAP_CUDA(cudaMemcpyAsync(e->h_dmax.p, p->max_dist_per_read, n * 4, cudaMemcpyHostToDevice,
                                  st),
                  "max_dist H2D");
        dp.max_dist_per_read = static_cast<const int32_t*>(e->h_dmax.p);
    }
    const uint8_t* d_reads = static_cast<const uint8_t*>(e->h_reads.p) - lo;
    rc = align_batch_device(idx, e, d_reads, static_cast<const uint64_t*>(e->h_offsets.p), n, &dp,
                            static_cast<snap_result*>(e->h_out.p), st, plain);
    if (rc) return rc;
    SNAP_CUDA(cudaMemcpyAsync(out, e->h_out.p, n * sizeof(snap_result), cudaMemcpyDeviceToHost, st),
              "results D2H");
    SNAP_CUDA(cudaStreamSynchronize(st), "snap_align");
    return SNAP_OK;
}

}  // namespace snapgpu

using namespace snapgpu;

extern "C" int snap_align(const snap_index* idx, const uint8_t* reads, const uint64_t* offsets,
                          uint64_t n, const snap_params* p, snap_result* out) {
    return align_host(idx, reads, offsets, n, p, out, false);
}

extern "C" int snap_align_plain(const snap_index* idx, const uint8_t* reads,
                                const uint64_t* offsets, uint64_t n, const snap_params* p,
                                snap_result* out) {
    return align_host(idx, reads, offsets, n, p, out, true);
}

extern "C" int snap_index_configure(snap_index* idx, int autotune, int cuda_graphs, int team) {
    clear_error();
    if (!idx) {
        set_error("snap_index_configure: index is NULL");
        return SNAP_E_INVAL;
    }
    if (team < -1 || team > 2) {
        set_error("snap_index_configure: team must be -1, 0, 1 or 2 (got %d)", team);
        return SNAP_E_INVAL;
    }
    std::lock_guard<std::mutex> lock(idx->engine->mu);
    idx->engine->autotune = autotune != 0;
    idx->engine->use_graphs = cuda_graphs != 0;
    idx->engine->team = team;
    if (!autotune) idx->engine->tuned.clear();
    return SNAP_OK;
}

extern "C" int snap_last_call_stats(const snap_index* idx, snap_call_stats* out) {
    clear_error();
    if (!idx || !out) {
        set_error("snap_last_call_stats: NULL argument");
        return SNAP_E_INVAL;
    }
    std::lock_guard<std::mutex> lock(idx->engine->mu);
    *out = idx->engine->last;
    return SNAP_OK;
}

extern "C" int snap_align_device(const snap_index* idx, const uint8_t* d_reads,
                                 const uint64_t* d_offsets, uint64_t n, const snap_params* p,
                                 snap_result* d_out, void* stream) {
    clear_error();
    if (!idx) {
        set_error("snap_align_device: index is NULL");
        return SNAP_E_INVAL;
    }
    std::lock_guard<std::mutex> lock(idx->engine->mu);
    return align_batch_device(idx, idx->engine, d_reads, d_offsets, n, p, d_out,
                              static_cast<cudaStream_t>(stream), false);
}

extern "C" int snap_align_plain_device(const snap_index* idx, const uint8_t* d_reads,
                                       const uint64_t* d_offsets, uint64_t n,
                                       const snap_params* p, snap_result* d_out, void* stream) {
    clear_error();
    if (!idx) {
        set_error("snap_align_plain_device: index is NULL");
        return SNAP_E_INVAL;
    }
    std::lock_guard<std::mutex> lock(idx->engine->mu);
    return align_batch_device(idx, idx->engine, d_reads, d_offsets, n, p, d_out,
                              static_cast<cudaStream_t>(stream), true);
}

// ---------------------------------------------------------------------------
// snap_align_device_noalloc: the batched form with no device allocation.
//
// Some callers cannot let a library call cudaMalloc/cudaFree: a framework that
// has already reserved the device memory for its own pool (an allocation would
// fail or fragment it), a serving thread that must never stall (cudaMalloc and
// cudaFree can synchronize the whole device), or a process whose device memory
// is audited through its own allocator.  For them this entry point keeps every
// piece of scratch (batch statistics, status word, queue heads, packed reads,
// the list of reads deferred to the second launch and the candidate tables that
// do not fit in shared memory) in one file-scope device array of fixed size that
// is created when the library's code is loaded onto a device and lives until the
// process exits.  The first launch fills every SM with warps that use shared-
// memory tables only and lists the rare read whose candidates outgrow them; a
// second launch aligns just the listed reads, one global table per warp.
// ---------------------------------------------------------------------------
namespace snapgpu {

constexpr size_t kNoAllocBytes = 64ull << 20;      // whole array: 64 MiB per device
constexpr size_t kNoAllocHeadBytes = 4096;         // statistics, status, counters, queue heads
constexpr size_t kNoAllocReadBytes = 48ull << 20;  // packed reads (4 bases per byte)
constexpr size_t kNoAllocDeferIds = 1u << 19;      // reads listed for the second launch
constexpr size_t kNoAllocTableBytes =
    kNoAllocBytes - kNoAllocHeadBytes - kNoAllocReadBytes - kNoAllocDeferIds * 4;
// head region: batch statistics, then at kNoAllocQueueOff the two launches' queue
// heads and the count of listed reads
constexpr size_t kNoAllocQueueOff = 1024;
static_assert(sizeof(BatchStats) <= kNoAllocQueueOff, "statistics overlap the queue heads");
static_assert(kNoAllocQueueOff + 3 * sizeof(unsigned long long) <= kNoAllocHeadBytes,
              "queue heads past the head region");
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device.  In host code the
// array's name only stands for the symbol, so the address is looked up once per
// device (with that device current) and cached.
static int noalloc_scratch(void** out) {
    int dev = 0;
    SNAP_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("snap_align_device_noalloc: device %d out of range", dev);
        return SNAP_E_INVAL;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            return cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                             "cudaGetSymbolAddress(scratch)");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return SNAP_OK;
}

static int align_noalloc(const snap_index* idx, const uint8_t* d_reads, const uint64_t* d_offsets,
                         uint64_t n, const snap_params* p, snap_result* d_out,
                         cudaStream_t stream) {
    const char* where = "snap_align_device_noalloc";
    int rc = validate_params(idx, p);
    if (rc) return rc;
    if (n == 0) return SNAP_OK;
    if (!d_reads || !d_offsets || !d_out) {
        set_error("%s: NULL buffer", where);
        return SNAP_E_INVAL;
    }
    if ((reinterpret_cast<uintptr_t>(d_offsets) | reinterpret_cast<uintptr_t>(d_out)) % 8 ||
        (p->max_dist_per_read && reinterpret_cast<uintptr_t>(p->max_dist_per_read) % 4)) {
        set_error("%s: offsets and results must be 8-byte aligned, max_dist_per_read 4-byte "
                  "aligned", where);
        return SNAP_E_INVAL;
    }
    void* base = nullptr;
    if ((rc = noalloc_scratch(&base))) return rc;
    unsigned char* b = static_cast<unsigned char*>(base);
    BatchStats* d_st = reinterpret_cast<BatchStats*>(b);
    unsigned long long* d_q = reinterpret_cast<unsigned long long*>(b + kNoAllocQueueOff);
    // d_q[0]: queue head of the first launch, [1]: of the second, [2]: reads listed
    uint32_t* d_words = reinterpret_cast<uint32_t*>(b + kNoAllocHeadBytes);
    uint32_t* d_defer = reinterpret_cast<uint32_t*>(b + kNoAllocHeadBytes + kNoAllocReadBytes);
    unsigned char* d_tables = b + kNoAllocHeadBytes + kNoAllocReadBytes + kNoAllocDeferIds * 4;

    // the array keeps the previous call's contents: clear what must start at zero
    SNAP_CUDA(cudaMemsetAsync(d_st, 0, sizeof(BatchStats), stream), "clear statistics");
    SNAP_CUDA(cudaMemsetAsync(d_q, 0, 3 * sizeof(unsigned long long), stream), "clear heads");
    int sms = 0, dev = 0;
    SNAP_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    SNAP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    k_read_stats<<<stats_grid(sms, n), kStatsThreads, 0, stream>>>(
        d_offsets, n, idx->s, idx->stride, p->num_seeds, p->max_dist, p->conf_diff, p->max_hits,
        p->max_dist_per_read, d_st);
    SNAP_CUDA(cudaGetLastError(), "stats launch");
    BatchStats hs;
    uint64_t base0 = 0;
    SNAP_CUDA(cudaMemcpyAsync(&hs, d_st, sizeof(hs), cudaMemcpyDeviceToHost, stream), "stats");
    SNAP_CUDA(cudaMemcpyAsync(&base0, d_offsets, sizeof(base0), cudaMemcpyDeviceToHost, stream),
              "offset");
    SNAP_CUDA(cudaStreamSynchronize(stream), where);
    if (hs.status) return status_to_code(hs.status, where);
    const uint64_t nwords = (hs.total_bases + kReadPadBases + 15) / 16 + 8;
    if (nwords * 4 > kNoAllocReadBytes) {
        set_error("%s: the batch has %llu bases; this entry point holds at most %llu bases "
                  "per call (split the batch or use snap_align_device)",
                  where, (unsigned long long)hs.total_bases,
                  (unsigned long long)((kNoAllocReadBytes / 4 - 8) * 16 + 15 - kReadPadBases -
                                       15));
        return SNAP_E_INVAL;
    }

    FusedArgs a;
    memset(&a, 0, sizeof(a));
    a.genome = idx->genome_words;
    a.G = idx->G;
    a.s = idx->s;
    a.slots = idx->slots;
    a.T = idx->T;
    a.positions = idx->positions;
    a.rwords = d_words;
    a.offsets = d_offsets;
    a.base0 = base0;
    a.order = nullptr;
    a.n_items = n;
    a.head = d_q;
    a.d_max = p->max_dist;
    a.h_max = p->max_hits;
    a.c = p->conf_diff;
    a.num_seeds = p->num_seeds;
    a.first_seeds = p->first_seeds;
    a.collapse = p->collapse_duplicates;
    a.stride = idx->stride;
    a.dmax_per_read = p->max_dist_per_read;
    shift_list(idx->s, a.shifts, &a.n_shifts);
    a.out = d_out;
    a.status = &d_st->status;
    a.ctr = &d_st->ctr;
    const int mmax = std::max(1u, hs.max_len);
    const int Lmax = std::max(0, hs.max_L0);
    const int nmax = std::max(1, hs.max_seeds);
    auto up4 = [](int w) { return (w + 3) & ~3; };
    a.wx = up4((mmax + 15) / 16 + 4);
    a.wt = up4((mmax + Lmax + 15 + 15) / 16 + 4);
    a.seed_cap = nmax;
    a.lv_ints = Lmax > 31 ? up4(2 * (2 * Lmax + 4)) : 0;
    const int fixed_words = 2 * a.wx + a.wt + 4 * a.seed_cap + a.lv_ints;
    int warps = 8;
    const int budget_words = 200 * 1024 / 4;
    while (warps > 1 && warps * (fixed_words + 7 * 64) > budget_words) warps >>= 1;
    int scap = 1024;
    while (scap > 64 && warps * (fixed_words + 7 * scap) > budget_words) scap >>= 1;
    a.scap = scap;
    a.off_xr = a.wx;
    a.off_tw = 2 * a.wx;
    a.off_seeds = a.off_tw + a.wt;
    a.off_tab = a.off_seeds + 4 * a.seed_cap;
    a.off_hits = a.off_tab + 4 * scap;
    a.off_dense = a.off_hits + 4 * (scap / 2);
    a.off_lv = a.off_dense + up4(scap / 2);
    a.warp_words = a.off_lv + a.lv_ints;
    const size_t smem = (size_t)warps * a.warp_words * 4;
    if (smem > 227 * 1024) {
        set_error("%s: read length %d needs too much shared memory", where, mmax);
        return SNAP_E_INVAL;
    }
    const FusedKernel kfn = fused_kernel_for(Lmax, false, param_variant(idx, p));
    if ((rc = raise_smem_limit((const void*)kfn, (size_t)(int)smem))) return rc;
    int per_sm = 0;
    SNAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, warps * 32, smem),
              "occupancy");
    if (per_sm < 1) per_sm = 1;
    uint64_t gcap = 64;
    while (gcap < 2 * hs.max_hits_bound) gcap <<= 1;
    if (gcap > kMaxTableSlots) {
        set_error("%s: seeds x max_hits per read (%llu) exceeds %u", where,
                  (unsigned long long)hs.max_hits_bound, kMaxTableSlots / 2);
        return SNAP_E_INVAL;
    }
    // global table of one warp (slots, hits, dense list) for the reads that need one
    const uint64_t per_warp = gcap * (sizeof(CandSlot) + sizeof(HitRec) / 2 + 2);
    const uint64_t max_table_warps = kNoAllocTableBytes / per_warp;
    const bool tables = gcap > (uint64_t)scap;  // some read may outgrow shared memory
    if (tables && max_table_warps < 1) {
        set_error("%s: seeds x max_hits per read (%llu) needs %llu bytes of candidate "
                  "table for one warp, more than the %llu this entry point holds (fewer seeds "
                  "or a smaller max_hits, or use snap_align_device)",
                  where, (unsigned long long)hs.max_hits_bound, (unsigned long long)per_warp,
                  (unsigned long long)kNoAllocTableBytes);
        return SNAP_E_INVAL;
    }
    const int aligned = ((reinterpret_cast<uintptr_t>(d_reads) + base0) % 16) == 0;
    k_pack_reads<<<grid_cap(sms, nwords, 256), 256, 0, stream>>>(
        d_reads, base0, hs.total_bases, d_words, nwords, aligned, &d_st->status);
    SNAP_CUDA(cudaGetLastError(), "pack launch");

    // first launch: every SM full of warps, shared-memory tables only; a read whose
    // candidates outgrow them is listed for the second launch
    const uint64_t blocks1 = std::min<uint64_t>((uint64_t)sms * per_sm, (n + warps - 1) / warps);
    if (tables) {
        a.defer_ids = d_defer;
        a.defer_count = d_q + 2;
        a.defer_cap = kNoAllocDeferIds;
    }
    kfn<<<(unsigned)std::max<uint64_t>(1, blocks1), warps * 32, smem, stream>>>(a);
    SNAP_CUDA(cudaGetLastError(), "align launch");
    int st = 0;
    unsigned long long ndefer = 0;
    SNAP_CUDA(cudaMemcpyAsync(&st, &d_st->status, sizeof(int), cudaMemcpyDeviceToHost, stream),
              "status");
    SNAP_CUDA(cudaMemcpyAsync(&ndefer, d_q + 2, sizeof(ndefer), cudaMemcpyDeviceToHost, stream),
              "listed reads");
    SNAP_CUDA(cudaStreamSynchronize(stream), where);
    if (st & kStTableFull) {
        set_error("%s: more than %llu reads of the batch need a candidate table larger than "
                  "shared memory (split the batch or use snap_align_device)",
                  where, (unsigned long long)kNoAllocDeferIds);
        return SNAP_E_INVAL;
    }
    if (st || ndefer == 0) return status_to_code(st, where);

    // second launch: the listed reads, as many warps as the array has tables for
    int warps2 = (int)std::min<uint64_t>((uint64_t)warps, max_table_warps);
    const uint64_t tw_cap = std::min<uint64_t>(max_table_warps, (uint64_t)sms * per_sm * warps2);
    uint64_t blocks2 = std::min<uint64_t>(tw_cap / warps2, (ndefer + warps2 - 1) / warps2);
    blocks2 = std::max<uint64_t>(1, blocks2);
    const uint64_t tw = blocks2 * warps2;
    a.defer_ids = nullptr;
    a.defer_count = nullptr;
    a.defer_cap = 0;
    a.order = d_defer;
    a.n_items = ndefer;
    a.head = d_q + 1;
    a.gtab = reinterpret_cast<CandSlot*>(d_tables);
    a.ghits = reinterpret_cast<HitRec*>(d_tables + tw * gcap * sizeof(CandSlot));
    a.gdense = reinterpret_cast<uint32_t*>(d_tables + tw * gcap * sizeof(CandSlot) +
                                           tw * (gcap / 2) * sizeof(HitRec));
    a.gcap = (uint32_t)gcap;
    // the array keeps the previous call's contents: empty the tables this launch uses
    k_init_ctab<<<grid_cap(sms, tw * gcap, 256), 256, 0, stream>>>(a.gtab, tw * gcap);
    SNAP_CUDA(cudaGetLastError(), "table init");
    kfn<<<(unsigned)blocks2, warps2 * 32, (size_t)warps2 * a.warp_words * 4, stream>>>(a);
    SNAP_CUDA(cudaGetLastError(), "align launch");
    SNAP_CUDA(cudaMemcpyAsync(&st, &d_st->status, sizeof(int), cudaMemcpyDeviceToHost, stream),
              "status");
    SNAP_CUDA(cudaStreamSynchronize(stream), where);
    return status_to_code(st, where);
}

}  // namespace snapgpu

extern "C" int snap_align_device_noalloc(const snap_index* idx, const uint8_t* d_reads,
                                         const uint64_t* d_offsets, uint64_t n,
                                         const snap_params* p, snap_result* d_out, void* stream) {
    clear_error();
    return align_noalloc(idx, d_reads, d_offsets, n, p, d_out, static_cast<cudaStream_t>(stream));
}
