// snap_plain.cu — the plain form of the alignment path: one kernel launch per
// stage over the whole batch, no persistent queue, no graph.  It computes the
// same results as the batched form by another route:
//   1. probe:      one thread per (read, probe) looks the seed up in the index
//                  (a seed is one probe, or k consecutive ones on a stride-k index);
//   2. scan:       per-read hit counts -> offsets (host reads the total);
//   3. candidates: one warp per read gathers the votes of its non-popular seeds
//                  into a per-read table (distinct (strand, p) keys) and records,
//                  in seed order, which table slot each hit went to;
//   4. distance:   one warp per candidate computes its edit distance once, at the
//                  largest limit the read can use, L0 = d_max + c - 1;
//   5. replay:     one warp per read replays Algorithm 1 seed by seed from the
//                  recorded votes, with ED(L) = (d0 <= L ? d0 : over) (and the
//                  seeds-first variant's deferred first pick).
// Step 5 gives Algorithm 1's result because the pick order depends only on the
// votes and on which candidates were scored, never on distances, and every
// limit the algorithm uses is at most L0, so the distance at any limit follows
// from the one at L0.
#include <algorithm>
#include <cstring>

#include "snap_device.cuh"
#include "snap_engine.h"
#include "snap_internal.h"
#include "snap_scan.cuh"

namespace snapgpu {

namespace {

constexpr int kInfP = 1 << 28;
constexpr unsigned long long kKeyMaskP = (1ull << 33) - 1;
constexpr uint32_t kNoSlot = 0xffffffffu;
constexpr uint32_t kScoredBit = 0x80000000u;

struct PlainArgs {
    const uint32_t* genome;
    uint64_t G;
    int s;
    const IndexSlot* slots;
    uint64_t T;
    const uint32_t* positions;
    const uint32_t* rwords;
    const uint64_t* offsets;
    uint64_t base0;
    uint64_t n;
    int nmax;  // seed slots per read
    int d_max, h_max, c, num_seeds;
    int first_seeds;  // seeds-first variant (<= 1: Algorithm 1)
    int stride;       // index stride: probes per seed
    const int32_t* dmax_per_read;
    uint8_t shifts[32];
    int n_shifts;
    SeedRec* seeds;           // [n][nmax]
    uint32_t* hits_per_read;  // [n]
    unsigned long long* hit_off;  // [n] exclusive scan of hits_per_read
    CandSlot* table;          // per read: 2 * hits slots at 2 * hit_off[r]
    uint32_t* events;         // per read: hits entries at hit_off[r]
    HitRec* hitlist;          // per read: hits entries at hit_off[r]
    unsigned long long* items;    // (read << 32) | slot
    unsigned long long* n_items;
    uint32_t* dense;          // per read: the used table slots, at hit_off[r]
    uint32_t* ndense;         // [n] number of used slots
    snap_result* out;
    int* status;
    DevCounters* ctr;
    // distance-stage shared memory per warp (words)
    int wx, wt, lv_ints, warp_words;
};

// seeds of a read of length m
__device__ __forceinline__ int read_seed_groups(const PlainArgs& a, int m) {
    if (m < a.s) return 0;
    int nn = a.num_seeds > 0 ? a.num_seeds : m / a.s;
    return min(nn, m - a.s + 1);
}

// probe slots of a read (stride-k index: k probes per seed)
__device__ __forceinline__ int read_seeds(const PlainArgs& a, int m) {
    return read_seed_groups(a, m) * a.stride;
}

__device__ __forceinline__ void add_counter(unsigned long long* dst, unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}

// 1. one thread per (read, seed slot)
__global__ void k_plain_probe(PlainArgs a) {
    const uint64_t total = a.n * (uint64_t)a.nmax;
    unsigned long long my_seeds = 0;
    uint32_t my_steps = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    // every thread of a warp runs the same number of iterations so the counter
    // reduction below is warp-converged
    const uint64_t iters = (total + stride - 1) / stride;
    for (uint64_t it = 0; it < iters; ++it) {
        const uint64_t t = it * stride + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
        if (t >= total) continue;
        const uint64_t r = t / a.nmax;
        const int i = (int)(t % a.nmax);
        const uint64_t o0 = a.offsets[r];
        const int m = (int)(a.offsets[r + 1] - o0);
        const int nn = read_seeds(a, m);
        SeedRec rec;
        rec.fwd_ref = rec.rc_ref = 0;
        rec.fwd_n = rec.rc_n = 0;
        rec.offset = 0;
        rec.flags = 0;
        rec.pad = 0;
        bool p0 = false;
        const int o = i < nn ? probe_offset(i, a.stride, m, a.s, a.shifts, a.n_shifts, &p0) : -1;
        if (o >= 0) {
            rec.flags = (uint8_t)(kSeedValid | (p0 ? kSeedPass0 : 0));
            rec.offset = (uint16_t)o;
            const uint64_t rb = o0 - a.base0 + kReadPadBases;
            const uint64_t v = get32(a.rwords, rb + (uint64_t)o) & kmer_mask(a.s);
            uint32_t cnt = 0;
            lookup_seed(a.slots, a.T, a.positions, v, a.s, &rec, &cnt, a.status, &my_steps);
            ++my_seeds;
            if (cnt > (uint32_t)a.h_max) {
                rec.flags |= kSeedPopular;
            } else if (rec.fwd_n + rec.rc_n) {
                atomicAdd(&a.hits_per_read[r], (uint32_t)rec.fwd_n + rec.rc_n);
            }
        }
        a.seeds[t] = rec;
    }
    add_counter(&a.ctr->seeds, my_seeds);
    add_counter(&a.ctr->slot_reads, my_steps);
}

__device__ __forceinline__ uint32_t table_insert_slot(CandSlot* tab, uint32_t cap,
                                                      unsigned long long key, int* status) {
    uint32_t h = (uint32_t)(mix64(key) % cap);
    for (uint32_t step = 0; step < cap; ++step) {
        const unsigned long long prev = atomicCAS(&tab[h].key, kEmptyKey, key);
        if (prev == kEmptyKey || prev == key) return h;
        h = (h + 1 == cap) ? 0 : h + 1;
    }
    atomicOr(status, kStTableFull);
    return kNoSlot;
}

// 3. one warp per read: distinct candidates and the slot of every hit
__global__ void k_plain_candidates(PlainArgs a) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long my_list = 0;
    for (uint64_t r = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; r < a.n;
         r += warps) {
        const uint32_t H = a.hits_per_read[r];
        if (H == 0) continue;
        const uint64_t base = a.hit_off[r];
        const uint32_t cap = 2 * H;
        CandSlot* tab = a.table + 2 * base;
        for (uint32_t j = lane; j < cap; j += 32) {
            CandSlot e;
            e.key = kEmptyKey;
            e.votes = 0;
            e.state = kUnscored;
            tab[j] = e;
        }
        __syncwarp();
        const uint64_t o0 = a.offsets[r];
        const int m = (int)(a.offsets[r + 1] - o0);
        const int nn = read_seeds(a, m);
        uint64_t cur = base;
        for (int i = 0; i < nn; ++i) {
            const SeedRec rec = a.seeds[r * a.nmax + i];
            if (rec.flags & kSeedPopular) continue;
            const int tot = (int)rec.fwd_n + rec.rc_n;
            const int o = rec.offset;
            for (int j = lane; j < tot; j += 32) {
                const bool fwd = j < rec.fwd_n;
                uint32_t l;
                if (rec.flags & kSeedFwdInline) {
                    l = fwd ? rec.fwd_ref : rec.rc_ref;
                } else {
                    l = fwd ? __ldg(a.positions + rec.fwd_ref + j)
                            : __ldg(a.positions + rec.rc_ref + (j - rec.fwd_n));
                    ++my_list;
                }
                const long long p = fwd ? (long long)l - o : (long long)l - (m - o - a.s);
                uint32_t slot = kNoSlot;
                if (p >= 0)
                    slot = table_insert_slot(tab, cap,
                                             2ull * (unsigned long long)p + (fwd ? 0 : 1),
                                             a.status);
                a.events[cur + j] = slot;
            }
            cur += tot;
        }
        __syncwarp();
        // one distance work item per distinct candidate, and the read's dense list
        uint32_t nd = 0;
        for (uint32_t j0 = 0; j0 < cap; j0 += 32) {
            const uint32_t j = j0 + lane;
            const bool used = j < cap && tab[j].key != kEmptyKey;
            const unsigned bal = __ballot_sync(kFull, used);
            unsigned long long at = 0;
            if (lane == 0 && bal) at = atomicAdd(a.n_items, (unsigned long long)__popc(bal));
            at = __shfl_sync(kFull, at, 0);
            if (used) {
                const unsigned rank = __popc(bal & ((1u << lane) - 1));
                a.items[at + rank] = (r << 32) | j;
                a.dense[base + nd + rank] = j;
            }
            nd += __popc(bal);
        }
        if (lane == 0) a.ndense[r] = nd;
    }
    add_counter(&a.ctr->list_entries, my_list);
}

// 4. one warp per candidate: distance at L0 = d_max + c - 1
__global__ void __launch_bounds__(256) k_plain_distance(PlainArgs a) {
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t* X = smem + (size_t)wib * a.warp_words;
    uint32_t* Tw = X + a.wx;
    int* lvA = a.lv_ints ? reinterpret_cast<int*>(Tw + a.wt) : nullptr;
    int* lvB = lvA ? lvA + a.lv_ints / 2 : nullptr;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned long long total = *a.n_items;
    unsigned long long calls = 0, over = 0, words = 0;
    for (uint64_t it = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; it < total;
         it += warps) {
        const unsigned long long item = a.items[it];
        const uint64_t r = item >> 32;
        const uint32_t slot = (uint32_t)(item & 0xffffffffu);
        CandSlot* cs = a.table + 2 * a.hit_off[r] + slot;
        const unsigned long long key = cs->key;
        const uint64_t o0 = a.offsets[r];
        const int m = (int)(a.offsets[r + 1] - o0);
        const int dmax = a.dmax_per_read ? a.dmax_per_read[r] : a.d_max;
        const int L0 = dmax + a.c - 1;
        const uint64_t rb = o0 - a.base0 + kReadPadBases;
        const int strand = (int)(key & 1);
        const uint64_t p = key >> 1;
        const int nw = (m + 15) / 16;
        for (int w = lane; w < nw + 3; w += 32) {
            uint32_t x = 0;
            if (w < nw) {
                x = strand ? rev_groups32(~get16(a.rwords, rb + (uint64_t)m - 16 - 16ull * w))
                           : get16(a.rwords, rb + 16ull * w);
            } else if (w == nw && !strand) {
                x = get16(a.rwords, rb + 16ull * w);
            }
            X[w] = x;
        }
        int d = kOver;
        int nwt = 0;
        if (L0 >= 0) {
            const int n_t = (int)min(a.G - p, (uint64_t)(m + L0));
            const uint64_t w0 = p >> 4;
            const int tb = (int)(p & 15);
            nwt = (tb + n_t + 15) / 16 + 2;
            for (int w = lane; w < nwt; w += 32) Tw[w] = __ldg(a.genome + w0 + w);
            __syncwarp();
            d = lv_warp(X, m, Tw, tb, n_t, L0, lane, lvA, lvB, a.status);
        }
        __syncwarp();
        if (lane == 0) {
            cs->state = d >= 0 ? d : kOver;
            calls++;
            over += (d < 0);
            words += (unsigned)nwt;
        }
    }
    if (lane == 0) {
        if (calls) atomicAdd(&a.ctr->ed_calls, calls);
        if (over) atomicAdd(&a.ctr->ed_over, over);
        if (words) atomicAdd(&a.ctr->window_words, words);
    }
}

__device__ __forceinline__ unsigned long long bucket_p(unsigned long long key) {
    return ((key >> 6) << 1) | (key & 1);
}

// 5. one warp per read: Algorithm 1 replayed from the recorded votes
__global__ void k_plain_replay(PlainArgs a) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t r = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; r < a.n;
         r += warps) {
        const uint64_t o0 = a.offsets[r];
        const int m = (int)(a.offsets[r + 1] - o0);
        const int nn = read_seeds(a, m);
        const int dmax = a.dmax_per_read ? a.dmax_per_read[r] : a.d_max;
        const int c = a.c;
        const uint32_t H = a.hits_per_read[r];
        const uint64_t base = H ? a.hit_off[r] : 0;
        const uint32_t cap = 2 * H;
        CandSlot* tab = a.table + 2 * base;
        HitRec* hits = a.hitlist + base;
        long long res_loc = -1;
        int res_d = -1, res_strand = 0, res_cls = SNAP_NOT_FOUND;
        if (nn > 0) {
            int d_best = kInfP, d_second = kInfP, nh = 0, t = 0;
            unsigned long long best_key = 0;
            bool any_nonpopular = false, returned = false;
            auto limit = [&]() -> int {
                if (d_best > dmax) return dmax + c - 1;
                if (d_second >= d_best + c) return d_best + c - 1;
                return d_best - 1;
            };
            const uint32_t nd = H ? a.ndense[r] : 0;
            const uint32_t* dense = a.dense + base;
            auto pick = [&]() -> unsigned long long {
                unsigned long long best = 0;
                for (uint32_t q = lane; q < nd; q += 32) {
                    const uint32_t j = dense[q];
                    const CandSlot e = tab[j];
                    // the table holds every seed's keys from the start; a key takes part
                    // only once a seed processed so far has voted for it
                    if (e.key != kEmptyKey && e.votes != 0 && !(e.votes & kScoredBit)) {
                        const unsigned long long v = ((unsigned long long)e.votes << 53) |
                                                     ((kKeyMaskP - e.key) << 20) | j;
                        best = v > best ? v : best;
                    }
                }
                return warp_max_u64(best);
            };
            auto score = [&](unsigned long long packed) {
                const uint32_t slot = (uint32_t)(packed & 0xfffffu);
                const unsigned long long key = kKeyMaskP - ((packed >> 20) & kKeyMaskP);
                const int L = limit();
                const int d0 = tab[slot].state;
                const int d = (L >= 0 && d0 >= 0 && d0 <= L) ? d0 : kOver;
                if (lane == 0) {
                    tab[slot].votes |= kScoredBit;
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
                        const unsigned long long bb = bucket_p(key);
                        int v = kInfP;
                        for (int j = lane; j < nh; j += 32) {
                            const HitRec h = hits[j];
                            if (bucket_p(h.key) != bb) v = min(v, h.d);
                        }
                        d_second = warp_min_i32(v);
                    } else if (bucket_p(key) != bucket_p(best_key)) {
                        d_second = min(d_second, d);
                    }
                }
            };
            // per seed, the probe after which a pick happens (its last non-popular
            // one), and the last such probe (seeds-first variant)
            int last_np = -1;
            const int ng = read_seed_groups(a, m);
            for (int g = lane; g < ng; g += 32)
                last_np = max(last_np, mark_seed_group(g, a.stride, nn, [&](int i) {
                                  return &a.seeds[r * a.nmax + i].flags;
                              }));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                last_np = max(last_np, __shfl_xor_sync(kFull, last_np, o));
            __syncwarp();
            int voted = 0;
            uint64_t cur = base;
            for (int i = 0; i < nn; ++i) {
                const SeedRec rec = a.seeds[r * a.nmax + i];
                if ((rec.flags & (kSeedValid | kSeedPopular)) != kSeedValid) continue;
                any_nonpopular = true;
                const int tot = (int)rec.fwd_n + rec.rc_n;
                for (int j = lane; j < tot; j += 32) {
                    const uint32_t slot = a.events[cur + j];
                    if (slot != kNoSlot) atomicAdd(&tab[slot].votes, 1u);
                }
                cur += tot;
                __syncwarp();
                if (rec.flags & kSeedCountT) ++t;
                if (!(rec.flags & kSeedPick)) continue;  // more probes of this seed to come
                if (++voted < a.first_seeds && i < last_np) continue;  // seeds-first
                const unsigned long long pk = cap ? pick() : 0ull;
                if (pk) score(pk);
                if (d_best < c && d_second < d_best + c) {
                    returned = true;
                    break;
                }
                if (t >= d_best + c) {
                    for (;;) {
                        const unsigned long long q = cap ? pick() : 0ull;
                        if (!q) break;
                        score(q);
                    }
                    break;
                }
            }
            if (!returned && d_best <= dmax && d_second >= d_best + c) {
                res_cls = SNAP_SINGLE_HIT;
            } else if (returned || d_best <= dmax || !any_nonpopular) {
                res_cls = SNAP_MULTIPLE_HITS;
            } else {
                res_cls = SNAP_NOT_FOUND;
            }
            if (res_cls != SNAP_NOT_FOUND && d_best <= dmax) {
                res_loc = (long long)(best_key >> 1);
                res_strand = (int)(best_key & 1);
                res_d = d_best;
            }
        }
        if (lane == 0) {
            unsigned long long* dst = reinterpret_cast<unsigned long long*>(a.out + r);
            dst[0] = (unsigned long long)res_loc;
            dst[1] = (unsigned long long)(uint32_t)res_d |
                     ((unsigned long long)((uint32_t)res_strand | ((uint32_t)res_cls << 8))
                      << 32);
        }
        __syncwarp();
    }
}

}  // namespace

int align_plain(const snap_index* idx, Engine* e, const uint64_t* d_offsets, uint64_t n,
                const snap_params* p, snap_result* d_out, cudaStream_t stream,
                const BatchPrep& bp) {
    int rc;
    PlainArgs a;
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
    a.n = n;
    a.nmax = std::max(1, bp.st.max_seeds);
    a.d_max = p->max_dist;
    a.h_max = p->max_hits;
    a.c = p->conf_diff;
    a.num_seeds = p->num_seeds;
    a.first_seeds = p->first_seeds;
    a.stride = idx->stride;
    a.dmax_per_read = p->max_dist_per_read;
    shift_list(idx->s, a.shifts, &a.n_shifts);
    a.out = d_out;
    BatchStats* d_st = static_cast<BatchStats*>(e->stats.p);
    a.status = &d_st->status;
    a.ctr = &d_st->ctr;
    if (bp.st.max_hits_bound * 2 > kMaxTableSlots) {
        set_error("snap_align_plain: seeds x max_hits per read (%llu) exceeds %u",
                  (unsigned long long)bp.st.max_hits_bound, kMaxTableSlots / 2);
        return SNAP_E_INVAL;
    }
    if (!e->pev[0])
        for (auto& ev : e->pev) SNAP_CUDA(cudaEventCreate(&ev), "event create");

    // 1. probe
    const uint64_t nseed = n * (uint64_t)a.nmax;
    if ((rc = e->p_seeds.ensure(nseed * sizeof(SeedRec), "seed records"))) return rc;
    if ((rc = e->p_hits.ensure(n * sizeof(uint32_t), "hit counts"))) return rc;
    if ((rc = e->p_hitoff.ensure(n * sizeof(unsigned long long), "hit offsets"))) return rc;
    if ((rc = e->p_partial.ensure(scan_blocks(n) * sizeof(unsigned long long) + 64, "scan")))
        return rc;
    if ((rc = e->p_misc.ensure(64, "counters"))) return rc;
    a.seeds = static_cast<SeedRec*>(e->p_seeds.p);
    a.hits_per_read = static_cast<uint32_t*>(e->p_hits.p);
    a.hit_off = static_cast<unsigned long long*>(e->p_hitoff.p);
    unsigned long long* misc = static_cast<unsigned long long*>(e->p_misc.p);
    a.n_items = misc;  // [0] item count, [1] hit total
    SNAP_CUDA(cudaMemsetAsync(a.hits_per_read, 0, n * sizeof(uint32_t), stream), "clear");
    SNAP_CUDA(cudaMemsetAsync(misc, 0, 64, stream), "clear");
    SNAP_CUDA(cudaEventRecord(e->pev[3], stream), "event");
    e->launches++;
    k_plain_probe<<<grid_cap(e->sms, nseed, 256), 256, 0, stream>>>(a);
    SNAP_CUDA(cudaGetLastError(), "probe launch");
    SNAP_CUDA(cudaEventRecord(e->pev[0], stream), "event");
    // 2. offsets of every read's hits
    e->launches += 3;
    exclusive_scan<uint32_t, unsigned long long, unsigned long long>(
        a.hits_per_read, a.hit_off, n, static_cast<unsigned long long*>(e->p_partial.p),
        misc + 1, stream);
    SNAP_CUDA(cudaGetLastError(), "scan launch");
    unsigned long long* h_tot = reinterpret_cast<unsigned long long*>(
        static_cast<char*>(e->pin.p) + 3072);
    SNAP_CUDA(cudaMemcpyAsync(h_tot, misc + 1, 8, cudaMemcpyDeviceToHost, stream), "total");
    SNAP_CUDA(cudaStreamSynchronize(stream), "snap_align_plain");
    const uint64_t Htot = std::max<unsigned long long>(1, *h_tot);
    if ((rc = e->p_table.ensure(2 * Htot * sizeof(CandSlot), "candidate tables"))) return rc;
    if ((rc = e->p_events.ensure(Htot * sizeof(uint32_t), "hit events"))) return rc;
    if ((rc = e->p_hitlist.ensure(Htot * sizeof(HitRec), "hit lists"))) return rc;
    if ((rc = e->p_items.ensure(Htot * sizeof(unsigned long long), "work items"))) return rc;
    if ((rc = e->p_dense.ensure(Htot * sizeof(uint32_t) + n * sizeof(uint32_t), "dense lists")))
        return rc;
    a.dense = static_cast<uint32_t*>(e->p_dense.p);
    a.ndense = a.dense + Htot;
    a.table = static_cast<CandSlot*>(e->p_table.p);
    a.events = static_cast<uint32_t*>(e->p_events.p);
    a.hitlist = static_cast<HitRec*>(e->p_hitlist.p);
    a.items = static_cast<unsigned long long*>(e->p_items.p);
    // 3. candidates
    e->launches++;
    k_plain_candidates<<<grid_cap(e->sms, n * 32, 256), 256, 0, stream>>>(a);
    SNAP_CUDA(cudaGetLastError(), "candidates launch");
    SNAP_CUDA(cudaEventRecord(e->pev[1], stream), "event");
    // 4. distances at L0 (one warp per candidate)
    const int mmax = std::max(1u, bp.st.max_len);
    const int Lmax = std::max(0, bp.st.max_L0);
    auto up4 = [](int w) { return (w + 3) & ~3; };
    a.wx = up4((mmax + 15) / 16 + 4);
    a.wt = up4((mmax + Lmax + 30) / 16 + 4);
    a.lv_ints = Lmax > 31 ? up4(2 * (2 * Lmax + 4)) : 0;
    a.warp_words = a.wx + a.wt + a.lv_ints;
    int warps = 8;
    while (warps > 1 && (size_t)warps * a.warp_words * 4 > 200 * 1024) warps >>= 1;
    const size_t smem = (size_t)warps * a.warp_words * 4;
    if (smem > 227 * 1024) {
        set_error("snap_align_plain: reads too long for the distance stage");
        return SNAP_E_INVAL;
    }
    if ((rc = raise_smem_limit((const void*)k_plain_distance, (size_t)(int)smem))) return rc;
    int per_sm = 1;
    SNAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_plain_distance,
                                                            warps * 32, smem),
              "occupancy");
    per_sm = std::max(1, per_sm);
    e->launches++;
    k_plain_distance<<<e->sms * per_sm, warps * 32, smem, stream>>>(a);
    SNAP_CUDA(cudaGetLastError(), "distance launch");
    SNAP_CUDA(cudaEventRecord(e->pev[2], stream), "event");
    // 5. replay
    e->launches++;
    k_plain_replay<<<grid_cap(e->sms, n * 32, 256), 256, 0, stream>>>(a);
    SNAP_CUDA(cudaGetLastError(), "replay launch");
    return SNAP_OK;
}

}  // namespace snapgpu
