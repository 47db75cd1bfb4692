// snap_light.cu — Algorithm 1 ("SNAP alignment algorithm") with one thread per
// short read, the first length bucket of the batched form.
//
// A read is handled here when it is short (m <= 128), uses at most 6 seeds, has a
// largest edit-distance limit d_max + c - 1 <= 15 and its non-popular seeds hit at
// most 8 index positions; the thread then runs the whole per-read loop alone:
// seed probes, votes in a small per-thread candidate list, the most-voted pick,
// the limit schedule, a Landau-Vishkin edit distance over one diagonal at a time,
// best / second best over 32-base buckets and the exits.  An edit distance that
// would need a fifth round is computed by the whole warp (see k_align_light).
// Any other read is appended to a device list that the warp-per-read kernel
// (snap_align.cu) drains next, starting from the probe records written here, so
// every result comes from exactly one of the two, with the same readings of the
// paper (see snap_align.cu).
//
// Per-thread arrays live in shared memory in column order (word w of thread t at
// w * blockDim + t) so that a warp's accesses to the same word fall in 32
// different banks.
#include <algorithm>
#include <cstring>

#include "snap_device.cuh"
#include "snap_engine.h"
#include "snap_internal.h"

namespace snapgpu {

constexpr int kLightMaxM = kLightBucketMaxM;
constexpr int kLightMaxL = kLightBucketMaxL;
// Index hits a read may have and stay here.  The per-thread candidate arrays live
// in local memory, whose footprint competes with shared memory for L1: 8 measured
// faster than 4, 6, 12, 16, 24 or 32 on both the 5%- and the 50%-repeat recipes
// (the warp kernel takes the rest).
constexpr int kLightMaxCands = 8;
// A thread posts its distance to the warp rather than start edit distance round 4
// (16 diagonals done): the rare long distances would otherwise hold the other 31
// lanes of the warp idle.
constexpr int kLightMaxRounds = 4;
constexpr int kLightXW = kLightMaxM / 16 + 2;                           // read words + 2
constexpr int kLightTW = (15 + kLightMaxM + kLightMaxL + 15) / 16 + 2;  // window words
constexpr int kLightRW = 2 * (kLightMaxRounds - 1) + 3;                 // diagonals + 2
constexpr int kLightWords = 2 * kLightXW + kLightTW + kLightRW;
// per warp: a read strand and a window for the distances the warp computes together
constexpr int kLightScratchWords = (kLightXW + kLightTW + 3) & ~3;

// shared memory of a block of `threads` threads
constexpr size_t light_smem_bytes(int threads) {
    return ((size_t)kLightWords * threads + (size_t)(threads / 32) * kLightScratchWords) * 4;
}

namespace {

constexpr int kInfL = 1 << 28;

struct LightArgs {
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
    int d_max, h_max, c, num_seeds;
    int first_seeds;
    int stride;  // index stride: probes per seed
    const int32_t* dmax_per_read;
    uint8_t shifts[32];
    int n_shifts;
    snap_result* out;
    uint32_t* heavy_ids;
    unsigned long long* heavy_count;
    SeedRec* hseeds;   // probe records of handed-over reads (kLightHandoverSlots per read)
    uint8_t* hprobed;  // per read: 1 when hseeds holds them
    int* status;
    DevCounters* ctr;
    DevCounters* ctr_light;
    BatchStats* stats;  // kernel start and end clocks
};

// 32 bases from a column-stored packed sequence (stride = threads per block)
__device__ __forceinline__ uint64_t col32(const uint32_t* col, int i, int st) {
    const int q = i >> 4;
    const uint32_t sh = (uint32_t)(i & 15) * 2u;
    const uint32_t w0 = col[q * st], w1 = col[(q + 1) * st], w2 = col[(q + 2) * st];
    return ((uint64_t)__funnelshift_r(w1, w2, sh) << 32) | __funnelshift_r(w0, w1, sh);
}

// VARIANT: the index has a stride > 1 or first_seeds > 1 (probe slots grouped
// per seed, picks deferred); without it a probe is a seed and every non-popular
// one picks, which keeps the common case's registers free.
//
// A thread first does everything that touches memory: its read, its seed
// probes, the candidates its non-popular seeds vote for (at most 8), and for
// each candidate an edit distance at the read's largest limit L0 = d_max + c - 1
// stopped before a fifth round.  It then runs Algorithm 1 on those results: the
// pick order depends only on the votes, and a distance at any limit L <= L0
// follows from the one at L0 (exact when d <= L, else over), so a candidate
// whose speculative distance came out exact needs no further work.  A candidate
// that needed a fifth round is over for any L <= 3; for a larger L the thread
// posts it and waits.  When every thread of the warp has ended or posted, the
// warp computes the posted distances one after another with all 32 lanes (one
// diagonal per lane) and the posting threads resume where they stopped.
template <bool VARIANT>
__global__ void __launch_bounds__(256, 5) k_align_light(LightArgs a) {
    extern __shared__ __align__(16) uint32_t smem[];
    const int tid = threadIdx.x, lane = tid & 31;
    const int st = blockDim.x;  // column stride of the per-thread arrays
    uint32_t* Xf = smem + tid;
    uint32_t* Xr = Xf + kLightXW * st;
    uint32_t* Tw = Xr + kLightXW * st;
    int* R = reinterpret_cast<int*>(Tw + kLightTW * st);
    // this warp's scratch for warp-wide distances: read strand, then window
    uint32_t* wscr = smem + kLightWords * st + (tid >> 5) * kLightScratchWords;
    const uint64_t r = blockIdx.x * (uint64_t)st + tid;
    if (tid == 0) atomicMax(&a.stats->light_start_ns_neg, ~globaltimer_ns());

    uint32_t c_seeds = 0, c_slots = 0, c_list = 0, c_ed = 0, c_over = 0, c_words = 0, c_done = 0;
    // the read and its Algorithm 1 state
    int m = 0, n = 0, dmax = 0;
    bool heavy = false;  // the warp-per-read kernel takes the read
    bool live = false;   // Algorithm 1 still running here
    constexpr int kLightMaxSeeds = VARIANT ? kLightVariantMaxSeeds : kLightBucketMaxSeeds;
    SeedRec seeds[kLightMaxSeeds];
    // candidates: key 2p + strand, the distance at L0 found up front (exact d,
    // kOver, or kLaneGaveUp when it needs a fifth round), votes, and the state
    // Algorithm 1 gave it (kUnscored, kOver or the distance)
    unsigned long long ckey[kLightMaxCands];
    int8_t csd[kLightMaxCands];
    uint8_t cvotes[kLightMaxCands];
    int8_t cstate[kLightMaxCands];
    // votes in seed order: the candidate of every vote, and where each probe slot's end
    uint8_t evc[kLightMaxCands];
    uint8_t evend[kLightMaxSeeds];
    // the hits are the scored candidates whose state is a distance (>= 0)
    int nc = 0, t = 0, voted = 0, i = 0, last_np = -1;
    int d_best = kInfL, d_second = kInfL;
    unsigned long long best_key = 0;
    bool any_nonpopular = false, returned = false, draining = false;
    int phase = 0;  // 0: next seed's votes, 1: pick and score, 2: exit tests
    // a distance posted to the warp: the candidate, its limit, and the result
    bool posted = false, resumed = false;
    int pend_pick = 0, pend_L = 0, pend_d = 0;
    const int c = a.c;

    if (r < a.n) {
        const uint64_t o0 = a.offsets[r];
        m = (int)(a.offsets[r + 1] - o0);
        const int s = a.s;
        int ng = 0;  // seeds
        if (m >= s) {
            ng = a.num_seeds > 0 ? a.num_seeds : m / s;
            ng = min(ng, m - s + 1);
        }
        const int stride = VARIANT ? a.stride : 1;
        n = ng * stride;  // probe slots (stride-k index: k per seed)
        dmax = a.dmax_per_read ? a.dmax_per_read[r] : a.d_max;
        heavy = m > kLightMaxM || n > kLightMaxSeeds || dmax + c - 1 > kLightMaxL;
        if (!heavy && n > 0) {
            const uint64_t rb = o0 - a.base0 + kReadPadBases;
            const int nw = (m + 15) / 16;
            // the read's aligned packed words (one before, one after) go to the
            // window column first; both strands are cut from them
            const uint64_t q0 = rb >> 4;
            const uint32_t sh = (uint32_t)(rb & 15) * 2u;
            const uint64_t xe = rb + (uint64_t)m;
            const int dq = (int)((xe >> 4) - q0);
            const uint32_t shx = (uint32_t)(xe & 15) * 2u;
            load_words_col(Tw, st, a.rwords, q0 - 1, nw + 2);
#pragma unroll
            for (int w = 0; w < kLightXW; ++w) {
                uint32_t f = 0, rc = 0;
                if (w < nw) {
                    f = __funnelshift_r(Tw[(w + 1) * st], Tw[(w + 2) * st], sh);
                    rc = rev_groups32(
                        ~__funnelshift_r(Tw[(dq - w) * st], Tw[(dq - w + 1) * st], shx));
                }
                Xf[w * st] = f;
                Xr[w * st] = rc;
            }
            // seed lookups
            unsigned H = 0;
            for (int q = 0; q < n; ++q) {
                bool p0 = false;
                const int o = VARIANT ? probe_offset(q, stride, m, s, a.shifts, a.n_shifts, &p0)
                                      : seed_offset(q, m, s, a.shifts, a.n_shifts, &p0);
                SeedRec rec;
                rec.pad = 0;
                if (o < 0) {  // a probe that does not fit in the read
                    rec.flags = 0;
                    rec.offset = 0;
                    rec.fwd_n = rec.rc_n = 0;
                    rec.fwd_ref = rec.rc_ref = 0;
                    seeds[q] = rec;
                    continue;
                }
                rec.flags = (uint8_t)(kSeedValid | (p0 ? kSeedPass0 : 0));
                rec.offset = (uint16_t)o;
                const uint64_t v = col32(Xf, o, st) & kmer_mask(s);
                uint32_t cnt = 0;
                lookup_seed(a.slots, a.T, a.positions, v, s, &rec, &cnt, a.status, &c_slots);
                ++c_seeds;
                if (cnt > (uint32_t)a.h_max) {
                    rec.flags |= kSeedPopular;
                } else {
                    H += (unsigned)rec.fwd_n + rec.rc_n;
                    if (stride == 1) {  // a probe is a seed
                        rec.flags |= (uint8_t)(kSeedPick | (p0 ? kSeedCountT : 0));
                        if (VARIANT) last_np = q;
                    }
                }
                seeds[q] = rec;
            }
            if (VARIANT && stride > 1)  // per seed: its last non-popular probe picks
                for (int g = 0; g < ng; ++g)
                    last_np = max(last_np, mark_seed_group(g, a.stride, n, [&](int q) {
                                      return &seeds[q].flags;
                                  }));
            heavy = H > (unsigned)kLightMaxCands;
            if (heavy && a.hseeds) {  // handed over after probing: the warp kernel
                for (int q = 0; q < n; ++q)  // starts from these records
                    a.hseeds[r * kLightHandoverSlots + q] = seeds[q];
                a.hprobed[r] = 1;
            }
            if (!heavy) {
                // the votes of every non-popular seed, in seed order, and the
                // distinct candidates they name
                int ne = 0;
                for (int q = 0; q < n; ++q) {
                    const SeedRec rec = seeds[q];
                    if ((rec.flags & (kSeedValid | kSeedPopular)) == kSeedValid) {
                        const int o = rec.offset;
                        const int tot = (int)rec.fwd_n + rec.rc_n;
                        for (int j = 0; j < tot; ++j) {
                            const bool fwd = j < rec.fwd_n;
                            uint32_t l;
                            if (rec.flags & kSeedFwdInline) {
                                l = fwd ? rec.fwd_ref : rec.rc_ref;
                            } else {
                                l = fwd ? __ldg(a.positions + rec.fwd_ref + j)
                                        : __ldg(a.positions + rec.rc_ref + (j - rec.fwd_n));
                                ++c_list;
                            }
                            const long long p =
                                fwd ? (long long)l - o : (long long)l - (m - o - s);
                            if (p < 0) continue;
                            const unsigned long long key =
                                2ull * (unsigned long long)p + (fwd ? 0 : 1);
                            int k = 0;
                            while (k < nc && ckey[k] != key) ++k;
                            if (k == nc) {
                                ckey[nc] = key;
                                cvotes[nc] = 0;
                                cstate[nc] = (int8_t)kUnscored;
                                ++nc;
                            }
                            evc[ne++] = (uint8_t)k;
                        }
                    }
                    evend[q] = (uint8_t)ne;
                }
                // every candidate's distance at L0, at most four rounds
                const int L0 = dmax + c - 1;
                for (int k = 0; k < nc; ++k) {
                    const unsigned long long key = ckey[k];
                    const uint64_t p = key >> 1;
                    const int n_t = (int)min(a.G - p, (uint64_t)(m + L0));
                    const int tb = (int)(p & 15);
                    const int nwt = (tb + n_t + 15) / 16 + 2;
                    load_words_col(Tw, st, a.genome, p >> 4, nwt);
                    c_words += nwt;
                    csd[k] = (int8_t)lv_lane((key & 1) ? Xr : Xf, st, m, Tw, st, tb, n_t, L0, R, st,
                                             kLightMaxRounds);
                }
                live = true;
            }
        }
    }

    for (;;) {
        // this thread: Algorithm 1 until the read ends or posts a long distance
        while (live && !posted) {
            if (phase == 0) {
                if (draining) {
                    phase = 1;
                } else {
                    while (i < n && (seeds[i].flags & (kSeedValid | kSeedPopular)) != kSeedValid)
                        ++i;
                    if (i >= n) {
                        live = false;
                        break;
                    }
                    const uint8_t flags = seeds[i].flags;
                    for (int e = i > 0 ? evend[i - 1] : 0; e < evend[i]; ++e) ++cvotes[evc[e]];
                    ++i;
                    any_nonpopular = true;
                    if (flags & kSeedCountT) ++t;
                    if (VARIANT) {
                        if (!(flags & kSeedPick)) continue;  // more probes of this seed
                        // seeds-first variant: no pick before first_seeds non-popular
                        // seeds (or all of them) have voted
                        if (++voted < a.first_seeds && i <= last_np) continue;
                    }
                    phase = 1;
                }
            }
            if (phase == 1) {
                int pick = -1, d = kOver;
                if (resumed) {  // the warp computed the distance this thread posted
                    resumed = false;
                    pick = pend_pick;
                    d = pend_d;
                } else {
                    // most-voted unscored candidate, ties to the smaller key (a
                    // candidate exists once some seed has voted for it)
                    for (int k = 0; k < nc; ++k) {
                        if (cstate[k] != kUnscored || cvotes[k] == 0) continue;
                        if (pick < 0 || cvotes[k] > cvotes[pick] ||
                            (cvotes[k] == cvotes[pick] && ckey[k] < ckey[pick]))
                            pick = k;
                    }
                    if (pick < 0 && draining) {
                        live = false;
                        break;
                    }
                    if (pick >= 0) {
                        int L;
                        if (d_best > dmax) {
                            L = dmax + c - 1;
                        } else if (d_second >= d_best + c) {
                            L = d_best + c - 1;
                        } else {
                            L = d_best - 1;
                        }
                        // the distance at L from the one found at L0 >= L
                        const int sd = csd[pick];
                        if (L < 0) {
                            d = kOver;
                        } else if (sd >= 0) {
                            d = sd <= L ? sd : kOver;
                        } else if (sd == kOver || L < kLightMaxRounds) {
                            d = kOver;  // over at L0, or needs more than L rounds
                        } else {        // needs a fifth round: the warp computes it
                            posted = true;
                            pend_pick = pick;
                            pend_L = L;
                            break;
                        }
                    }
                }
                if (pick >= 0) {
                    const unsigned long long key = ckey[pick];
                    ++c_ed;
                    c_over += (d < 0);
                    cstate[pick] = (int8_t)(d >= 0 ? d : kOver);
                    if (d >= 0) {
                        const unsigned long long bk = ((key >> 6) << 1) | (key & 1);
                        if (d < d_best) {
                            d_best = d;
                            best_key = key;
                            d_second = kInfL;
                            for (int k = 0; k < nc; ++k) {
                                if (cstate[k] < 0) continue;  // not a hit
                                const unsigned long long hb =
                                    ((ckey[k] >> 6) << 1) | (ckey[k] & 1);
                                if (hb != bk) d_second = min(d_second, (int)cstate[k]);
                            }
                        } else if (bk != (((best_key >> 6) << 1) | (best_key & 1))) {
                            d_second = min(d_second, d);
                        }
                    }
                }
                phase = 2;
            }
            if (phase == 2) {
                if (!draining) {
                    if (d_best < c && d_second < d_best + c) {
                        returned = true;
                        live = false;
                        break;
                    }
                    if (t >= d_best + c) draining = true;
                }
                phase = 0;
            }
        }
        // the warp: every posted distance, all lanes on each (limits are <= 15)
        const unsigned pm = __ballot_sync(kFull, posted);
        if (!pm) break;
        for (unsigned mm = pm; mm; mm &= mm - 1) {
            const int j = __ffs(mm) - 1;
            const unsigned long long key = __shfl_sync(kFull, posted ? ckey[pend_pick] : 0ull, j);
            const int L = __shfl_sync(kFull, pend_L, j);
            const int mj = __shfl_sync(kFull, m, j);
            const uint64_t p = key >> 1;
            const int n_t = (int)min(a.G - p, (uint64_t)(mj + L));
            const int tb = (int)(p & 15);
            const int nwt = (tb + n_t + 15) / 16 + 2;
            const uint32_t* Xj = smem + ((key & 1) ? kLightXW * st : 0) + (tid - lane + j);
            const uint32_t* gw = a.genome + (p >> 4);
            for (int w = lane; w < kLightXW + nwt; w += 32)
                wscr[w] = w < kLightXW ? Xj[w * st] : __ldg(gw + (w - kLightXW));
            if (lane == 0) c_words += nwt;
            __syncwarp();
            const int d = lv_warp_reg<1>(wscr, mj, wscr + kLightXW, tb, n_t, L, lane);
            __syncwarp();
            if (lane == j) {
                pend_d = d;
                posted = false;
                resumed = true;
            }
        }
    }

    if (r < a.n) {
        if (heavy) {
            const unsigned long long at = atomicAdd(a.heavy_count, 1ull);
            a.heavy_ids[at] = (uint32_t)r;
        } else {
            ++c_done;
            long long res_loc = -1;
            int res_d = -1, res_strand = 0, res_cls = SNAP_NOT_FOUND;
            if (n > 0) {
                if (!returned && d_best <= dmax && d_second >= d_best + c) {
                    res_cls = SNAP_SINGLE_HIT;
                } else if (returned || d_best <= dmax || !any_nonpopular) {
                    res_cls = SNAP_MULTIPLE_HITS;
                }
                if (res_cls != SNAP_NOT_FOUND && d_best <= dmax) {
                    res_loc = (long long)(best_key >> 1);
                    res_strand = (int)(best_key & 1);
                    res_d = d_best;
                }
            }
            unsigned long long* dst = reinterpret_cast<unsigned long long*>(a.out + r);
            dst[0] = (unsigned long long)res_loc;
            dst[1] = (unsigned long long)(uint32_t)res_d |
                     ((unsigned long long)((uint32_t)res_strand | ((uint32_t)res_cls << 8))
                      << 32);
        }
    }
    // seeds, slot_reads, list_entries, ed_calls, ed_over, window_words, -, reads_done
    unsigned long long v[8] = {c_seeds, c_slots, c_list, c_ed, c_over, c_words, 0, c_done};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(kFull, v[k], o);
    }
    if (lane == 0) {
        unsigned long long* dst = &a.ctr->seeds;
        unsigned long long* dl = &a.ctr_light->seeds;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (v[k]) {
                atomicAdd(dst + k, v[k]);
                atomicAdd(dl + k, v[k]);
            }
    }
    __syncthreads();
    if (tid == 0) atomicMax(&a.stats->light_end_ns, globaltimer_ns());
}

}  // namespace

// Shared-memory limit of the thread-per-read kernel, set once (before any capture).
int light_prepare() {
    int rc = raise_smem_limit((const void*)k_align_light<false>, light_smem_bytes(256));
    if (rc) return rc;
    return raise_smem_limit((const void*)k_align_light<true>, light_smem_bytes(256));
}

// Launch the thread-per-read bucket over all n reads; reads it does not take
// are appended to heavy_ids (count in *heavy_count, cleared here).
int launch_light(const snap_index* idx, Engine* e, const uint64_t* d_offsets, uint64_t n,
                 const snap_params* p, snap_result* d_out, cudaStream_t stream,
                 const BatchPrep& bp, uint32_t* heavy_ids, unsigned long long* heavy_count,
                 int threads, SeedRec* hseeds, uint8_t* hprobed) {
    LightArgs a;
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
    a.d_max = p->max_dist;
    a.h_max = p->max_hits;
    a.c = p->conf_diff;
    a.num_seeds = p->num_seeds;
    a.first_seeds = p->first_seeds;
    a.stride = idx->stride;
    a.dmax_per_read = p->max_dist_per_read;
    shift_list(idx->s, a.shifts, &a.n_shifts);
    a.out = d_out;
    a.heavy_ids = heavy_ids;
    a.heavy_count = heavy_count;
    a.hseeds = hseeds;
    a.hprobed = hprobed;
    BatchStats* d_st = static_cast<BatchStats*>(e->stats.p);
    a.status = &d_st->status;
    a.ctr = &d_st->ctr;
    a.ctr_light = &d_st->ctr_light;
    a.stats = d_st;
    if (threads != 64 && threads != 128 && threads != 256) threads = 128;
    const size_t smem = light_smem_bytes(threads);
    SNAP_CUDA(cudaMemsetAsync(heavy_count, 0, sizeof(unsigned long long), stream), "clear");
    const uint64_t blocks = (n + threads - 1) / threads;
    e->launches++;
    if (a.stride > 1 || a.first_seeds > 1)
        k_align_light<true><<<(unsigned)blocks, threads, smem, stream>>>(a);
    else
        k_align_light<false><<<(unsigned)blocks, threads, smem, stream>>>(a);
    SNAP_CUDA(cudaGetLastError(), "light launch");
    return SNAP_OK;
}

}  // namespace snapgpu
