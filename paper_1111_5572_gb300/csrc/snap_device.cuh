// snap_device.cuh — device helpers of the SNAP kernels: 2-bit packing,
// canonical s-mers, the index probe and the warp-cooperative bounded edit
// distance (farthest reach per diagonal).
#pragma once

#include <cstdint>

#include "snap_internal.h"

namespace snapgpu {

constexpr unsigned kFull = 0xffffffffu;

// A=0 C=1 G=2 T=3 from ASCII, by bits 1 and 2 of the letter (valid for the
// four uppercase letters only; is_acgt() checks).
__device__ __forceinline__ uint32_t code_of(uint32_t c) { return ((c >> 1) ^ (c >> 2)) & 3u; }
__device__ __forceinline__ bool is_acgt(uint32_t c) {
    return c == 'A' || c == 'C' || c == 'G' || c == 'T';
}

// Bases are packed 16 per 32-bit word, base i at bits 2*(i%16) of word i/16.
// 16 bases starting at any base index (the array is padded by one word).
__device__ __forceinline__ uint32_t get16(const uint32_t* w, uint64_t i) {
    const uint64_t q = i >> 4;
    return __funnelshift_r(w[q], w[q + 1], (uint32_t)(i & 15) * 2u);
}

// 32 bases starting at any base index (padded by two words).
__device__ __forceinline__ uint64_t get32(const uint32_t* w, uint64_t i) {
    const uint64_t q = i >> 4;
    const uint32_t sh = (uint32_t)(i & 15) * 2u;
    const uint32_t w0 = w[q], w1 = w[q + 1], w2 = w[q + 2];
    const uint32_t lo = __funnelshift_r(w0, w1, sh);
    const uint32_t hi = __funnelshift_r(w1, w2, sh);
    return ((uint64_t)hi << 32) | lo;
}

// Reverse the order of the 2-bit groups of a word.
__device__ __forceinline__ uint32_t rev_groups32(uint32_t x) {
    const uint32_t r = __brev(x);
    return ((r >> 1) & 0x55555555u) | ((r & 0x55555555u) << 1);
}
__device__ __forceinline__ uint64_t rev_groups64(uint64_t x) {
    const uint64_t r = __brevll(x);
    return ((r >> 1) & 0x5555555555555555ull) | ((r & 0x5555555555555555ull) << 1);
}

// Reverse complement of an s-mer held in the low 2s bits (complement of
// code x is 3 - x = x ^ 3, i.e. bitwise NOT).
__device__ __forceinline__ uint64_t kmer_revcomp(uint64_t v, int s) {
    return rev_groups64(~v) >> (64 - 2 * s);
}

__device__ __forceinline__ uint64_t kmer_mask(int s) {
    return s >= 32 ? ~0ull : ((1ull << (2 * s)) - 1ull);
}

// murmur3's 64-bit finaliser (a bijection), then a multiply-high to [0, T).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}
__device__ __forceinline__ IndexSlot load_slot(const IndexSlot* slots, uint64_t i) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(slots) + i);
    IndexSlot s;
    s.key = ((unsigned long long)v.y << 32) | v.x;
    s.field = v.z;
    s.nA = (uint16_t)(v.w & 0xffffu);
    s.nB = (uint16_t)(v.w >> 16);
    return s;
}

// The index table is a sequence of 64-byte buckets of four slots (T is a
// multiple of 4).  A key lives in its home bucket mulhi(mix(key), T/4) or, when
// that bucket was full at insertion, in the next non-full bucket; slots of a
// bucket fill in order, so an empty slot ends a lookup.  For seeds of at most 31
// bases (keys below 2^62) the top bit of a bucket's first key says whether some
// key whose home is this bucket spilled into a later one: a full home bucket
// without that bit ends the lookup of a key it does not hold.
constexpr int kBucketSlots = 4;
constexpr unsigned long long kSpillBit = 1ull << 63;
__host__ __device__ constexpr bool spill_flags(int s) { return s <= 31; }

__device__ __forceinline__ uint64_t home_bucket(uint64_t key, uint64_t T) {
    return __umul64hi(mix64(key), T / kBucketSlots);
}

// Probe for canonical key K.  Returns true and the slot when present.  Sets
// kStProbeRunaway in *status if the probe does not end within the table (a full
// table; cannot happen at load <= 2/3).  *steps counts slots read.
__device__ __forceinline__ bool probe_index(const IndexSlot* slots, uint64_t T, uint64_t K,
                                            IndexSlot* out, int* status, uint32_t* steps,
                                            bool flagged) {
    const uint64_t nb = T / kBucketSlots;
    uint64_t b = home_bucket(K, T);
    for (uint64_t step = 0; step < nb; ++step) {
        const uint4* q = reinterpret_cast<const uint4*>(slots) + b * kBucketSlots;
        uint4 v[kBucketSlots];
#pragma unroll
        for (int j = 0; j < kBucketSlots; ++j) v[j] = __ldg(q + j);
        *steps += kBucketSlots;
        bool empty = false;
        const unsigned long long first = ((unsigned long long)v[0].y << 32) | v[0].x;
#pragma unroll
        for (int j = 0; j < kBucketSlots; ++j) {
            unsigned long long key = ((unsigned long long)v[j].y << 32) | v[j].x;
            empty |= (key == kEmptyKey);
            if (j == 0 && flagged) key &= ~kSpillBit;
            if (key == K) {
                out->key = key;
                out->field = v[j].z;
                out->nA = (uint16_t)(v[j].w & 0xffffu);
                out->nB = (uint16_t)(v[j].w >> 16);
                return true;
            }
        }
        if (empty) return false;
        if (step == 0 && flagged && !(first & kSpillBit)) return false;  // none spilled
        b = (b + 1 == nb) ? 0 : b + 1;
    }
    atomicOr(status, kStProbeRunaway);
    return false;
}

// The seed lookups of one seed with forward s-mer v: the forward occurrences
// of v (strand-0 votes) and of revcomp(v) (strand-1 votes), from the
// canonical slot.  Fills everything of `rec` but offset/flags bits 1.
__device__ __forceinline__ void lookup_seed(const IndexSlot* slots, uint64_t T,
                                            const uint32_t* /*positions*/, uint64_t v, int s,
                                            SeedRec* rec, uint32_t* count, int* status,
                                            uint32_t* steps) {
    const uint64_t rc = kmer_revcomp(v, s);
    const bool pal = (v == rc);
    const bool v_is_key = (v <= rc);
    const uint64_t K = v_is_key ? v : rc;
    IndexSlot sl;
    rec->fwd_ref = rec->rc_ref = 0;
    rec->fwd_n = rec->rc_n = 0;
    *count = 0;
    if (!probe_index(slots, T, K, &sl, status, steps, spill_flags(s))) return;
    const uint32_t nA = sl.nA, nB = sl.nB;
    // where A and B start: inline when nA + nB == 1
    const bool single = (nA + nB) == 1;
    const uint32_t a_ref = sl.field, b_ref = single ? sl.field : sl.field + nA;
    uint32_t fn, rn, fr, rr;
    if (pal) {  // both lookups are the A list
        fn = rn = nA;
        fr = rr = a_ref;
    } else if (v_is_key) {
        fn = nA; fr = a_ref;
        rn = nB; rr = b_ref;
    } else {
        fn = nB; fr = b_ref;
        rn = nA; rr = a_ref;
    }
    *count = fn + rn;
    rec->fwd_n = (uint16_t)(fn > 65535u ? 65535u : fn);
    rec->rc_n = (uint16_t)(rn > 65535u ? 65535u : rn);
    rec->fwd_ref = fr;
    rec->rc_ref = rr;
    if (single) rec->flags |= (uint8_t)(kSeedFwdInline | kSeedRcInline);
}

// Offset of seed i of a read of length m (seed order: the non-overlapping
// pass, then the passes shifted by the entries of `shifts`).
__device__ __forceinline__ int seed_offset(int i, int m, int s, const uint8_t* shifts,
                                           int n_shifts, bool* pass0) {
    for (int q = 0; q < n_shifts; ++q) {
        const int d = shifts[q];
        const int cnt = (m - s - d >= 0) ? (m - s - d) / s + 1 : 0;
        if (i < cnt) {
            *pass0 = (d == 0);
            return d + i * s;
        }
        i -= cnt;
    }
    *pass0 = false;
    return -1;
}

// Probe slot i of a read for an index of windows starting at multiples of
// `stride` (1 = every window): seed i / stride of the order above, looked up at
// its offset + i % stride so that an error-free seed meets one indexed window
// whatever the alignment; -1 when that probe does not fit in the read.
__device__ __forceinline__ int probe_offset(int i, int stride, int m, int s,
                                            const uint8_t* shifts, int n_shifts, bool* pass0) {
    const int g = stride == 1 ? i : i / stride;
    const int j = i - g * stride;
    const int o = seed_offset(g, m, s, shifts, n_shifts, pass0);
    if (o < 0 || o + j + s > m) return -1;
    return o + j;
}

// Marks, for the probes of seed g (slots g*stride .. g*stride+stride-1 of
// flags), the last valid non-popular probe with kSeedPick (the seed's votes are
// in after it) and, when the seed is of the unshifted pass and none of its
// valid probes was popular, also kSeedCountT (it counts toward t).  Returns
// that probe's slot, or -1 when the seed has no non-popular probe.
template <typename FlagAt>
__device__ __forceinline__ int mark_seed_group(int g, int stride, int nslots, FlagAt flag_at) {
    int last = -1;
    bool all_np = true, p0 = false;
    for (int j = 0; j < stride; ++j) {
        const int i = g * stride + j;
        if (i >= nslots) break;
        const uint8_t f = *flag_at(i);
        if (!(f & kSeedValid)) continue;
        p0 = (f & kSeedPass0) != 0;
        if (f & kSeedPopular) {
            all_np = false;
        } else {
            last = i;
        }
    }
    if (last >= 0) *flag_at(last) |= (uint8_t)(kSeedPick | ((all_np && p0) ? kSeedCountT : 0));
    return last;
}

// ---- bounded edit distance -------------------------------------------------
// ED(X, T) = min over prefixes T[0..j) of Lev(X, T[0..j)), exact when <= L,
// else kOver.  X: m bases packed at X (padded); T: n bases packed at Tw from
// base index tb (padded).  Farthest reach per diagonal k = j - i, one round per
// distance e = 0..L (Landau-Vishkin); each lane keeps D consecutive diagonals
// in registers, neighbours across lanes by shuffles.  Runs on a full warp.

__device__ __forceinline__ int slide(const uint32_t* X, int m, const uint32_t* Tw, int tb, int n,
                                     int r, int k) {
    for (;;) {
        const int lim = min(m - r, n - (r + k));
        if (lim <= 0) return r;
        const uint32_t x = get16(X, (uint64_t)r) ^ get16(Tw, (uint64_t)(tb + r + k));
        const int adv = x ? ((__ffs(x) - 1) >> 1) : 16;
        if (adv >= lim) return r + lim;
        r += adv;
        if (adv < 16) return r;
    }
}

// 16 bases starting at base i of a packed sequence whose word w sits at w * stride.
__device__ __forceinline__ uint32_t get16s(const uint32_t* w, int i, int stride) {
    const int q = i >> 4;
    return __funnelshift_r(w[q * stride], w[(q + 1) * stride], (uint32_t)(i & 15) * 2u);
}

// The same distance computed by one thread: rounds e = 0..L, diagonals k = -e..e
// in increasing order, updated in place in R (round e-1's value is only read for
// |k| <= e-1, so R needs no initialisation).  X and T are packed at word strides
// xs and ts.  Returns kLaneGaveUp instead of starting round max_rounds (a caller
// that hands costly reads elsewhere); R holds 2 min(L, max_rounds - 1) + 3 values
// at stride rs, 32-bit, or 16-bit (RT = int16_t) for reads shorter than 2^14 bases
// and L < 2^13 (an invalid diagonal then stays negative through its increments).
constexpr int kLaneGaveUp = -3;
template <typename RT = int>
__device__ __forceinline__ int lv_lane(const uint32_t* X, int xs, int m, const uint32_t* Tw, int ts,
                                       int tb, int n, int L, RT* R, int rs,
                                       int max_rounds = 0x7fffffff) {
    constexpr int NEG = sizeof(RT) == 2 ? -0x4000 : -0x40000000;
    if (L < 0) return kOver;
    const int off = min(L, max_rounds - 1) + 1;  // R index of diagonal k is k + off
    for (int e = 0; e <= L; ++e) {
        if (e >= max_rounds) return kLaneGaveUp;
        int left_old = NEG;
        for (int k = -e; k <= e; ++k) {
            RT* slot = R + (k + off) * rs;
            const int cur_old = (k >= -(e - 1) && k <= e - 1) ? *slot : NEG;
            int r;
            if (e == 0) {
                r = 0;
            } else {
                const int right_old = (k + 1 <= e - 1) ? slot[rs] : NEG;
                r = max(max(cur_old + 1, right_old + 1), left_old);
            }
            left_old = cur_old;
            if (r > m) r = m;
            if (r + k > n) r = n - k;
            if (r < 0 || r + k < 0) {
                *slot = (RT)NEG;
                continue;
            }
            for (;;) {
                const int lim = min(m - r, n - (r + k));
                if (lim <= 0) break;
                const uint32_t x = get16s(X, r, xs) ^ get16s(Tw, tb + r + k, ts);
                const int adv = x ? ((__ffs(x) - 1) >> 1) : 16;
                if (adv >= lim) {
                    r += lim;
                    break;
                }
                r += adv;
                if (adv < 16) break;
            }
            *slot = (RT)r;
            if (r >= m) return e;
        }
    }
    return kOver;
}

template <int D>
__device__ inline int lv_warp_reg(const uint32_t* X, int m, const uint32_t* Tw, int tb, int n, int L,
                           int lane) {
    constexpr int NEG = -0x40000000;
    int R[D];
#pragma unroll
    for (int t = 0; t < D; ++t) R[t] = NEG;
    for (int e = 0; e <= L; ++e) {
        int left = __shfl_up_sync(kFull, R[D - 1], 1);
        int right = __shfl_down_sync(kFull, R[0], 1);
        if (lane == 0) left = NEG;
        if (lane == 31) right = NEG;
        int Rn[D];
        bool done = false;
#pragma unroll
        for (int t = 0; t < D; ++t) {
            const int k = lane * D + t - L;
            int r = NEG;
            if (k >= -e && k <= e) {
                if (e == 0) {
                    r = 0;
                } else {
                    const int rkm1 = (t == 0) ? left : R[t - 1];
                    const int rkp1 = (t == D - 1) ? right : R[t + 1];
                    r = max(max(R[t] + 1, rkp1 + 1), rkm1);
                }
                if (r > m) r = m;
                if (r + k > n) r = n - k;
                if (r < 0 || r + k < 0) {
                    r = NEG;
                } else {
                    r = slide(X, m, Tw, tb, n, r, k);
                    done |= (r >= m);
                }
            }
            Rn[t] = r;
        }
#pragma unroll
        for (int t = 0; t < D; ++t) R[t] = Rn[t];
        if (__any_sync(kFull, done)) return e;
    }
    return kOver;
}

// Same recurrence with the diagonals in shared memory (any L); Ra/Rb hold
// 2L+3 ints each.
__device__ inline int lv_warp_smem(const uint32_t* X, int m, const uint32_t* Tw, int tb, int n, int L,
                            int lane, int* Ra, int* Rb) {
    constexpr int NEG = -0x40000000;
    const int W = 2 * L + 3, off = L + 1;
    for (int i = lane; i < W; i += 32) {
        Ra[i] = NEG;
        Rb[i] = NEG;
    }
    __syncwarp();
    for (int e = 0; e <= L; ++e) {
        bool done = false;
        for (int idx = lane; idx < 2 * e + 1; idx += 32) {
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
        __syncwarp();
        if (__any_sync(kFull, done)) return e;
        int* t = Ra;
        Ra = Rb;
        Rb = t;
    }
    return kOver;
}

// Up to L = 31 the diagonals live in registers (one or two per lane).  Beyond,
// the shared-memory form spreads each round's 2e+1 active diagonals over all
// lanes, which beats walking several register diagonals per lane every round.
// Ra/Rb (2L+3 ints each) are required when L > 31; without them the call flags
// kStInternal and reports kOver.
__device__ __forceinline__ int lv_warp(const uint32_t* X, int m, const uint32_t* Tw, int tb, int n,
                                       int L, int lane, int* Ra, int* Rb, int* status) {
    if (L < 0) return kOver;
    if (L <= 15) return lv_warp_reg<1>(X, m, Tw, tb, n, L, lane);
    if (L <= 31) return lv_warp_reg<2>(X, m, Tw, tb, n, L, lane);
    if (Ra == nullptr) {
        if (lane == 0) atomicOr(status, kStInternal);
        return kOver;
    }
    return lv_warp_smem(X, m, Tw, tb, n, L, lane, Ra, Rb);
}

// Words [w0, w0 + nw) of `src` (nw <= 13; src 16-byte aligned) into the column
// dst[0], dst[st], ... with the 16-byte chunks that cover them loaded first, all
// at once, so the copy costs one memory round trip rather than one per word.
// The chunks end at most 3 words past w0 + nw - 1 (callers' arrays are padded).
__device__ __forceinline__ void load_words_col(uint32_t* dst, int st, const uint32_t* src,
                                               uint64_t w0, int nw) {
    const uint64_t a0 = w0 & ~3ull;
    const int sh = (int)(w0 - a0);
    const int nchunks = (sh + nw + 3) >> 2;
    const uint4* s4 = reinterpret_cast<const uint4*>(src + a0);
    uint4 v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = j < nchunks ? __ldg(s4 + j) : make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t wj[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = 4 * j + q - sh;
            if (k >= 0 && k < nw) dst[k * st] = wj[q];
        }
    }
}

// The device's global nanosecond clock.
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Warp-wide max of a 64-bit value.
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(kFull, v, o);
        v = w > v ? w : v;
    }
    return v;
}

__device__ __forceinline__ int warp_min_i32(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

}  // namespace snapgpu
