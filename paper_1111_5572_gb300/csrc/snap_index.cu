// snap_index.cu — device build of the SNAP seed index.
//
// What is indexed follows the "Hash Index" subsection: every overlapping s-mer
// of the genome (window slid one base at a time), and item 2 of the list after
// Algorithm 1 (both the forward and the reverse-complement version of each
// string can be found).  The layout is this library's own: one
// open-addressing table keyed by the canonical s-mer min(S, revcomp(S)) with
// the two orientations kept as separate position lists (so a 32-bit position
// never loses a bit to a strand flag), positions of keys seen once stored in
// the slot itself; slots are grouped in 64-byte buckets of four so that a
// lookup is normally one DRAM access.  Built count-then-fill with atomics; no
// sort.
#include <chrono>
#include <cstdio>

#include "snap_device.cuh"
#include "snap_internal.h"
#include "snap_scan.cuh"

namespace snapgpu {

// pack 16 ASCII bases per word; flags non-ACGT bytes
__global__ void k_pack_genome(const uint8_t* __restrict__ ascii, uint64_t G,
                              uint32_t* __restrict__ words, uint64_t nwords, int* status) {
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < nwords;
         w += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t b0 = w * 16;
        uint32_t word = 0;
        bool bad = false;
        if (b0 + 16 <= G) {
            const uint4 v = *reinterpret_cast<const uint4*>(ascii + b0);
            const uint32_t parts[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t c = (parts[q] >> (8 * j)) & 0xffu;
                    bad |= !is_acgt(c);
                    word |= code_of(c) << (2 * (4 * q + j));
                }
            }
        } else if (b0 < G) {
            for (uint64_t j = 0; b0 + j < G; ++j) {
                const uint32_t c = ascii[b0 + j];
                bad |= !is_acgt(c);
                word |= code_of(c) << (2 * j);
            }
        }
        words[w] = word;
        if (bad) atomicOr(status, kStBadBase);
    }
}

__global__ void k_init_slots(IndexSlot* slots, uint64_t T) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < T;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint4 v;
        v.x = v.y = 0xffffffffu;  // key = kEmptyKey
        v.z = v.w = 0;            // counts of the two orientations
        reinterpret_cast<uint4*>(slots)[i] = v;
    }
}

__device__ __forceinline__ void canonical_at(const uint32_t* words, uint64_t l, int s,
                                             uint64_t* K, int* orient) {
    const uint64_t v = get32(words, l) & kmer_mask(s);
    const uint64_t rc = kmer_revcomp(v, s);
    *K = v <= rc ? v : rc;
    *orient = v <= rc ? 0 : 1;  // palindromes count as orientation 0
}

// count pass: insert the canonical key of every indexed window (starts that are
// multiples of `stride`, 1 = every window) and count its orientation
__global__ void k_insert(const uint32_t* __restrict__ words, uint64_t npos, int s, int stride,
                         IndexSlot* slots, uint64_t T, int* status) {
    const uint64_t nidx = (npos + stride - 1) / stride;
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < nidx;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t l = q * (uint64_t)stride;
        uint64_t K;
        int o;
        canonical_at(words, l, s, &K, &o);
        const uint64_t nb = T / kBucketSlots;
        uint64_t b = home_bucket(K, T);
        bool placed = false;
        for (uint64_t step = 0; step < nb && !placed; ++step) {
            for (int j = 0; j < kBucketSlots; ++j) {
                const uint64_t i = b * kBucketSlots + j;
                unsigned long long* kp = &slots[i].key;
                unsigned long long cur = *reinterpret_cast<volatile unsigned long long*>(kp);
                if (cur == kEmptyKey) cur = atomicCAS(kp, kEmptyKey, (unsigned long long)K);
                if (cur == kEmptyKey || cur == K) {
                    uint32_t* cnt = reinterpret_cast<uint32_t*>(&slots[i].field) + o;
                    atomicAdd(cnt, 1u);
                    placed = true;
                    break;
                }
            }
            b = (b + 1 == nb) ? 0 : b + 1;
        }
        if (!placed) atomicOr(status, kStTableFull);
    }
}

// list length of every slot (0 for empty, singletons and keys too frequent to
// ever pass an h_max <= kListMax); counts distinct keys
__global__ void k_list_lengths(const IndexSlot* slots, uint64_t T, uint32_t* lens,
                               unsigned long long* distinct) {
    unsigned long long mine = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < T;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 v = reinterpret_cast<const uint4*>(slots)[i];
        const bool used = !(v.x == 0xffffffffu && v.y == 0xffffffffu);
        const uint64_t tot = (uint64_t)v.z + v.w;
        lens[i] = (used && tot >= 2 && tot <= kListMax) ? (uint32_t)tot : 0u;
        mine += used ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(kFull, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(distinct, mine);
}

// rewrite {key, countA, countB} as {key, start-or-0, sat16(countA), sat16(countB)}
__global__ void k_finalize_slots(IndexSlot* slots, uint64_t T, const uint32_t* starts) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < T;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint4 v = reinterpret_cast<uint4*>(slots)[i];
        if (v.x == 0xffffffffu && v.y == 0xffffffffu) continue;
        const uint32_t a = v.z, b = v.w;
        const uint64_t tot = (uint64_t)a + b;
        const uint32_t a16 = a > 65535u ? 65535u : a, b16 = b > 65535u ? 65535u : b;
        v.z = (tot >= 2 && tot <= kListMax) ? starts[i] : 0u;
        v.w = a16 | (b16 << 16);
        reinterpret_cast<uint4*>(slots)[i] = v;
    }
}

// fill pass for one orientation: A lists first (orient 0), then B (orient 1),
// so that B entries land after all A entries of their key
__global__ void k_fill(const uint32_t* __restrict__ words, uint64_t npos, int s, int stride,
                       IndexSlot* slots, uint64_t T, uint32_t* cursor, uint32_t* positions,
                       int which, int* status) {
    const uint64_t nidx = (npos + stride - 1) / stride;
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < nidx;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t l = q * (uint64_t)stride;
        uint64_t K;
        int o;
        canonical_at(words, l, s, &K, &o);
        if (o != which) continue;
        const uint64_t nb = T / kBucketSlots;
        uint64_t b = home_bucket(K, T);
        bool found = false, ended = false;
        for (uint64_t step = 0; step < nb && !found && !ended; ++step) {
            for (int j = 0; j < kBucketSlots; ++j) {
                const uint64_t i = b * kBucketSlots + j;
                const uint4 v = reinterpret_cast<const uint4*>(slots)[i];
                const uint64_t key = ((uint64_t)v.y << 32) | v.x;
                if (key == K) {
                    const uint32_t tot = (v.w & 0xffffu) + (v.w >> 16);
                    if (tot == 1) {
                        slots[i].field = (uint32_t)l;
                    } else if (tot <= kListMax) {
                        const uint32_t at = atomicAdd(&cursor[i], 1u);
                        positions[at] = (uint32_t)l;
                    }
                    found = true;
                    break;
                }
                if (key == kEmptyKey) {
                    ended = true;
                    break;
                }
            }
            b = (b + 1 == nb) ? 0 : b + 1;
        }
        if (!found) atomicOr(status, kStInternal);
    }
}

// After every key is placed: for each key that sits outside its home bucket, set
// kSpillBit on the home bucket's first key (that bucket is full, so its first
// slot holds a key; keys of s <= 31 bases never use the bit).
__global__ void k_mark_spills(IndexSlot* slots, uint64_t T) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < T;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long key =
            *reinterpret_cast<volatile unsigned long long*>(&slots[i].key);
        if (key == kEmptyKey) continue;
        const uint64_t h = home_bucket(key & ~kSpillBit, T);
        if (h != i / kBucketSlots) atomicOr(&slots[h * kBucketSlots].key, kSpillBit);
    }
}

static int grid_for(uint64_t n, int threads) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t want = (n + threads - 1) / threads;
    uint64_t cap = (uint64_t)sms * 32;
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    return (int)want;
}

}  // namespace snapgpu

using namespace snapgpu;

extern "C" int snap_index_build(const uint8_t* genome_ascii, uint64_t genome_len, int seed_len,
                                snap_index** out) {
    return snap_index_build_stride(genome_ascii, genome_len, seed_len, 1, out);
}

extern "C" int snap_index_build_stride(const uint8_t* genome_ascii, uint64_t genome_len,
                                       int seed_len, int stride, snap_index** out) {
    clear_error();
    std::lock_guard<std::recursive_mutex> lock(capture_alloc_mutex());
    if (!out) {
        set_error("snap_index_build: out is NULL");
        return SNAP_E_INVAL;
    }
    *out = nullptr;
    if (!genome_ascii) {
        set_error("snap_index_build: genome is NULL");
        return SNAP_E_INVAL;
    }
    if (seed_len < 8 || seed_len > 32) {
        set_error("snap_index_build: seed_len %d outside [8, 32]", seed_len);
        return SNAP_E_INVAL;
    }
    if (stride < 1 || stride > kMaxStride) {
        set_error("snap_index_build: stride %d outside [1, %d]", stride, kMaxStride);
        return SNAP_E_INVAL;
    }
    if (genome_len < (uint64_t)seed_len || genome_len >= (1ull << 32) - (1ull << 16)) {
        set_error("snap_index_build: genome_len %llu outside [seed_len, 2^32 - 2^16)",
                  (unsigned long long)genome_len);
        return SNAP_E_INVAL;
    }
    const auto t0 = std::chrono::steady_clock::now();
    snap_index* idx = new snap_index();
    cudaGetDevice(&idx->device);
    idx->G = genome_len;
    idx->s = seed_len;
    idx->stride = stride;
    const uint64_t npos = genome_len - seed_len + 1;
    const uint64_t nidx = (npos + stride - 1) / stride;  // indexed windows
    idx->T = ((nidx + nidx / 2 + 64) + kBucketSlots - 1) / kBucketSlots * kBucketSlots;  // load <= 2/3
    idx->genome_words_n = (genome_len + 15) / 16 + 8;

    uint8_t* d_ascii = nullptr;
    uint32_t* d_cursor = nullptr;
    int* d_status = nullptr;
    unsigned long long* d_counters = nullptr;  // [0] distinct, [1] scan total
    unsigned long long* d_partial = nullptr;
    cudaStream_t st = nullptr;

    auto fail = [&](int code) {
        cudaFree(d_ascii);
        cudaFree(d_cursor);
        cudaFree(d_status);
        cudaFree(d_counters);
        cudaFree(d_partial);
        cudaFree(idx->genome_words);
        cudaFree(idx->slots);
        cudaFree(idx->positions);
        if (st) cudaStreamDestroy(st);
        delete idx;
        return code;
    };
#define TRY(call, what)                                  \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return fail(cuda_fail(e_, what)); \
    } while (0)

    TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream create");
    TRY(cudaMalloc(&d_status, sizeof(int)), "status alloc");
    TRY(cudaMemsetAsync(d_status, 0, sizeof(int), st), "status clear");
    TRY(cudaMalloc(&d_counters, 2 * sizeof(unsigned long long)), "counter alloc");
    TRY(cudaMemsetAsync(d_counters, 0, 2 * sizeof(unsigned long long), st), "counter clear");
    TRY(cudaMalloc(&d_ascii, genome_len + 16), "genome staging alloc");
    TRY(cudaMemcpyAsync(d_ascii, genome_ascii, genome_len, cudaMemcpyHostToDevice, st),
        "genome copy");
    TRY(cudaMalloc(&idx->genome_words, idx->genome_words_n * 4), "packed genome alloc");
    TRY(cudaMemsetAsync(idx->genome_words, 0, idx->genome_words_n * 4, st), "packed clear");
    const uint64_t nw = (genome_len + 15) / 16;
    k_pack_genome<<<grid_for(nw, 256), 256, 0, st>>>(d_ascii, genome_len, idx->genome_words, nw,
                                                      d_status);
    TRY(cudaGetLastError(), "pack launch");
    int hstatus = 0;
    TRY(cudaMemcpyAsync(&hstatus, d_status, sizeof(int), cudaMemcpyDeviceToHost, st), "status");
    TRY(cudaStreamSynchronize(st), "pack");
    if (hstatus & kStBadBase) {
        set_error("snap_index_build: genome has a byte other than A, C, G, T");
        return fail(SNAP_E_INVAL);
    }
    cudaFree(d_ascii);
    d_ascii = nullptr;

    TRY(cudaMalloc(&idx->slots, idx->T * sizeof(IndexSlot)), "table alloc");
    k_init_slots<<<grid_for(idx->T, 256), 256, 0, st>>>(idx->slots, idx->T);
    k_insert<<<grid_for(nidx, 256), 256, 0, st>>>(idx->genome_words, npos, seed_len, stride,
                                                  idx->slots, idx->T, d_status);
    TRY(cudaGetLastError(), "insert launch");
    TRY(cudaMalloc(&d_cursor, idx->T * sizeof(uint32_t)), "cursor alloc");
    k_list_lengths<<<grid_for(idx->T, 256), 256, 0, st>>>(idx->slots, idx->T, d_cursor,
                                                          d_counters);
    TRY(cudaMalloc(&d_partial, sizeof(unsigned long long) * scan_blocks(idx->T)), "scan alloc");
    exclusive_scan<uint32_t, uint32_t, unsigned long long>(d_cursor, d_cursor, idx->T, d_partial,
                                                           d_counters + 1, st);
    TRY(cudaGetLastError(), "scan launch");
    k_finalize_slots<<<grid_for(idx->T, 256), 256, 0, st>>>(idx->slots, idx->T, d_cursor);
    unsigned long long hc[2] = {0, 0};
    TRY(cudaMemcpyAsync(hc, d_counters, sizeof(hc), cudaMemcpyDeviceToHost, st), "counters");
    TRY(cudaMemcpyAsync(&hstatus, d_status, sizeof(int), cudaMemcpyDeviceToHost, st), "status");
    TRY(cudaStreamSynchronize(st), "count pass");
    if (hstatus) {
        set_error("snap_index_build: table insert failed (status 0x%x)", hstatus);
        return fail(SNAP_E_INTERNAL);
    }
    idx->distinct = hc[0];
    idx->n_positions = hc[1];
    TRY(cudaMalloc(&idx->positions, (idx->n_positions + 4) * sizeof(uint32_t)), "list alloc");
    for (int which = 0; which < 2; ++which) {
        k_fill<<<grid_for(nidx, 256), 256, 0, st>>>(idx->genome_words, npos, seed_len, stride,
                                                    idx->slots, idx->T, d_cursor, idx->positions,
                                                    which, d_status);
    }
    TRY(cudaGetLastError(), "fill launch");
    if (spill_flags(seed_len)) {
        k_mark_spills<<<grid_for(idx->T, 256), 256, 0, st>>>(idx->slots, idx->T);
        TRY(cudaGetLastError(), "mark launch");
    }
    TRY(cudaMemcpyAsync(&hstatus, d_status, sizeof(int), cudaMemcpyDeviceToHost, st), "status");
    TRY(cudaStreamSynchronize(st), "fill pass");
    if (hstatus) {
        set_error("snap_index_build: fill failed (status 0x%x)", hstatus);
        return fail(SNAP_E_INTERNAL);
    }
    cudaFree(d_cursor);
    cudaFree(d_partial);
    cudaFree(d_status);
    cudaFree(d_counters);
    cudaStreamDestroy(st);
#undef TRY
    idx->device_bytes = idx->genome_words_n * 4 + idx->T * sizeof(IndexSlot) +
                        (idx->n_positions + 4) * sizeof(uint32_t);
    idx->engine = engine_create();
    idx->build_seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = idx;
    return SNAP_OK;
}

extern "C" int snap_index_free(snap_index* idx) {
    clear_error();
    if (!idx) return SNAP_OK;
    std::lock_guard<std::recursive_mutex> lock(capture_alloc_mutex());
    if (idx->engine) engine_destroy(idx->engine);
    cudaFree(idx->genome_words);
    cudaFree(idx->slots);
    cudaFree(idx->positions);
    delete idx;
    return SNAP_OK;
}

extern "C" int snap_index_info_get(const snap_index* idx, snap_index_info* out) {
    clear_error();
    if (!idx || !out) {
        set_error("snap_index_info_get: NULL argument");
        return SNAP_E_INVAL;
    }
    out->genome_len = idx->G;
    out->seed_len = idx->s;
    out->stride = idx->stride;
    out->table_slots = idx->T;
    out->distinct_seeds = idx->distinct;
    out->list_entries = idx->n_positions;
    out->device_bytes = idx->device_bytes;
    out->build_seconds = idx->build_seconds;
    return SNAP_OK;
}
