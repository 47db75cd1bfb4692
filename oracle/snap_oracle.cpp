// snap_oracle.cpp — plain, slow, CPU-only SNAP (Zaharia et al., arXiv 1111.5572).
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
// cpu_baseline / reference legs may load this library.  It shares no code,
// header, table or helper with the CUDA path (paper_1111_5572_gb300/); the two
// meet only at the seeded inputs from synth/.
//
// What it computes, and the passage each part follows:
//   * index: the "Hash Index" subsection — every overlapping s-mer of the genome
//     (sliding window of one base; or every k-th, R9), with lookups of both a seed and its reverse
//     complement, as "populate the index with both forward and reverse
//     complement versions" (item 2 of the list after Algorithm 1) asks.  Here it
//     is a sorted array of (s-mer, position) pairs searched with binary search.
//   * seed order: item 3 of that list — sequential non-overlapping seeds, then
//     shifts of s/2, then s/4, 3s/4, and so on.
//   * edit distance: the "Local Alignment" subsection — Ukkonen's O(nd) method
//     in its farthest-reach-per-diagonal (Landau-Vishkin) form, returning a
//     special value once d exceeds d_limit.  The textbook O(n^2) table is kept
//     beside it as the pin.
//   * per-read loop: Algorithm 1 ("SNAP alignment algorithm"), with the
//     32-base bucket merge of item 1 of the list after it.
//
// Readings taken where the paper is silent:
//   R1 count(S) = occurrences of S + occurrences of revcomp(S).  A forward
//      occurrence of S at l votes for (strand 0, p = l - o); an occurrence of
//      revcomp(S) at l votes for (strand 1, p = l - (m - o - s)), where o is the
//      seed offset and m the read length.  Candidates with p < 0 are dropped.
//   R2 seed shifts: 0, then floor(j*s/2^k) for k = 1, 2, ... and odd j < 2^k,
//      skipping repeats; each shift d gives offsets d, d+s, ... while o+s <= m.
//      The first n offsets are the seeds; n = floor(m/s) when not given.  The
//      "non-overlapping seeds tested" counter t counts shift-0 seeds whose
//      lookup was not skipped for popularity.
//   R3 EditDistance(Read, Reference[p], L) = min over e >= 0 of
//      Lev(X, G[p..p+e)) (start anchored at p, end free), X = read for strand 0
//      and its reverse complement for strand 1; exact when <= L, else "over".
//      Reference bases past the genome end do not exist (never match).
//   R4 pick = unscored candidate with the most votes, ties to the smaller key
//      2p+strand.  A candidate becomes scored even when its distance is over
//      the limit; such results are not hits.
//   R5 bucket merge: bucket = (strand, floor(p/32)); d_best = min over hits,
//      best = the earliest-scored hit reaching it; d_second = min over hits in
//      another bucket than best's.
//   R6 drain: when t >= d_best + c, score every remaining candidate in pick
//      order (limits recomputed, no early return inside), then stop seeding.
//      The exit tests run after every non-popular seed even if nothing was
//      left to score.
//   R7 result fields: single -> (p, strand, d_best); multiple -> best's
//      (p, strand, d_best) when d_best <= d_max, else (-1, 0, -1);
//      not found -> (-1, 0, -1).  "All seeds had > h_max entries" needs at
//      least one seed; a read shorter than s is not found.
//   R8 seeds-first variant (Local Alignment, the remark after the Baeza-Yates
//      test that looking up more seeds before scoring the first candidate was
//      tried): with first_seeds = k > 1, the first k non-popular seeds (all of
//      them when there are fewer) add their votes before the first pick;
//      from then on one pick per non-popular seed as in Algorithm 1.  No exit
//      test can pass before the first score, so none is skipped.
//   R9 stride-k index (Hash Index, Overlapping Seeds footnote: a window slid k
//      bases at a time gives a k-times smaller index and more lookups): only
//      positions l with l % k == 0 are indexed, and each seed of the R2 order
//      at offset o is looked up at o, o+1, ..., o+k-1 (those that fit), so an
//      error-free seed meets exactly one indexed position whatever the
//      alignment.  A probe is popular on its own count (indexed occurrences);
//      a seed votes with its non-popular probes and is skipped when all are
//      popular; it counts toward t (pass 0 seeds tested) only when none of its
//      probes was popular, since a skipped probe may be the one that meets the
//      index.  With k = 1 a probe is a seed and this is Algorithm 1.
#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstring>
#include <map>
#include <thread>
#include <utility>
#include <vector>

namespace {

constexpr int kInf = 1 << 28;  // "infinity" for d_best / d_second; sums stay far from overflow

int code_of(uint8_t ch) {
    switch (ch) {
        case 'A': return 0;
        case 'C': return 1;
        case 'G': return 2;
        case 'T': return 3;
        default: return -1;
    }
}

// s-mer value, first base most significant
uint64_t kmer_value(const uint8_t* codes, int s) {
    uint64_t v = 0;
    for (int j = 0; j < s; ++j) v = (v << 2) | codes[j];
    return v;
}

struct OracleIndex {
    int s = 0;
    int stride = 1;  // R9: only positions l with l % stride == 0 are indexed
    uint64_t G = 0;
    std::vector<uint8_t> genome;                            // codes 0..3
    std::vector<std::pair<uint64_t, uint32_t>> entries;     // (s-mer, position), sorted
    bool filtered = false;

    // positions l with G[l..l+s) == the s-mer `key`, ascending
    std::pair<size_t, size_t> range(uint64_t key) const {
        auto lo = std::lower_bound(entries.begin(), entries.end(), std::make_pair(key, (uint32_t)0));
        auto hi = std::upper_bound(entries.begin(), entries.end(),
                                   std::make_pair(key, (uint32_t)UINT32_MAX));
        return {size_t(lo - entries.begin()), size_t(hi - entries.begin())};
    }
};

// Seed offsets in the order of reading R2.
void seed_offsets(int m, int s, int n, std::vector<int>& offs, std::vector<uint8_t>& pass0) {
    offs.clear();
    pass0.clear();
    if (m < s || s <= 0) return;
    std::vector<int> shifts;
    std::vector<bool> used(s, false);
    shifts.push_back(0);
    used[0] = true;
    for (int k = 1; (int)shifts.size() < s && k < 62; ++k) {
        for (long long j = 1; j < (1LL << k); j += 2) {
            int d = (int)((j * s) >> k);
            if (!used[d]) {
                used[d] = true;
                shifts.push_back(d);
            }
        }
    }
    for (int d : shifts) {
        for (int o = d; o + s <= m; o += s) {
            offs.push_back(o);
            pass0.push_back(d == 0 ? 1 : 0);
        }
    }
    if (n < 0) n = 0;
    if ((int)offs.size() > n) {
        offs.resize(n);
        pass0.resize(n);
    }
}

// Bounded edit distance of reading R3 by farthest reach per diagonal.
// x: pattern codes (length m); t: text codes (length n).  Returns the distance
// when it is <= L, else -1.
int ed_lv(const uint8_t* x, int m, const uint8_t* t, int n, int L) {
    if (L < 0) return -1;
    const int NEG = INT_MIN / 4;
    const int W = 2 * L + 3, off = L + 1;  // diagonal k lives at index k + off, k in [-L-1, L+1]
    std::vector<int> prev(W, NEG), cur(W, NEG);
    for (int e = 0; e <= L; ++e) {
        std::fill(cur.begin(), cur.end(), NEG);
        for (int k = -e; k <= e; ++k) {
            int r;
            if (e == 0) {
                r = 0;
            } else {
                r = std::max(prev[k + off] + 1, prev[k + 1 + off] + 1);  // substitution, deletion
                r = std::max(r, prev[k - 1 + off]);                      // insertion
            }
            if (r > m) r = m;
            if (r + k > n) r = n - k;
            if (r < 0 || r + k < 0) continue;
            while (r < m && r + k < n && x[r] == t[r + k]) ++r;
            cur[k + off] = r;
            if (r == m) return e;
        }
        std::swap(prev, cur);
    }
    return -1;
}

// Textbook table: D[i][j] = Lev(x[0..i), t[0..j)); answer min_j D[m][j].
int ed_dp(const uint8_t* x, int m, const uint8_t* t, int n) {
    std::vector<int> row(n + 1), nxt(n + 1);
    for (int j = 0; j <= n; ++j) row[j] = j;
    for (int i = 1; i <= m; ++i) {
        nxt[0] = i;
        for (int j = 1; j <= n; ++j) {
            int sub = row[j - 1] + (x[i - 1] != t[j - 1] ? 1 : 0);
            int del = row[j] + 1;
            int ins = nxt[j - 1] + 1;
            nxt[j] = std::min(sub, std::min(del, ins));
        }
        std::swap(row, nxt);
    }
    return *std::min_element(row.begin(), row.end());
}

struct Params {
    int d_max, h_max, c, n_seeds;
    int first_seeds;  // <= 1: Algorithm 1; k > 1: the seeds-first variant (R8)
};

struct ReadResult {
    int64_t location;
    int32_t edit_distance;
    uint8_t strand;
    uint8_t cls;
};

struct Stats {
    uint64_t reads = 0, seeds_looked_up = 0, seeds_popular = 0, ed_calls = 0, ed_over = 0,
             ed_calls_after_first = 0, ed_over_after_first = 0, reads_with_hit = 0,
             first_scored_is_best = 0, candidates = 0;
    uint64_t cls[3] = {0, 0, 0};
    void add(const Stats& o) {
        reads += o.reads;
        seeds_looked_up += o.seeds_looked_up;
        seeds_popular += o.seeds_popular;
        ed_calls += o.ed_calls;
        ed_over += o.ed_over;
        ed_calls_after_first += o.ed_calls_after_first;
        ed_over_after_first += o.ed_over_after_first;
        reads_with_hit += o.reads_with_hit;
        first_scored_is_best += o.first_scored_is_best;
        candidates += o.candidates;
        for (int i = 0; i < 3; ++i) cls[i] += o.cls[i];
    }
};

enum { kNotFound = 0, kSingle = 1, kMultiple = 2 };

// One read through Algorithm 1.  mode 0: literal (EditDistance called with
// the limit of the moment).  mode 1: every candidate scored once up front at
// L0 = d_max + c - 1, then the same loop replayed with
// ED(L) = (d0 <= L ? d0 : over).
ReadResult align_one(const OracleIndex& idx, const uint8_t* ascii, int m, const Params& P,
                     int mode, Stats& st) {
    const int s = idx.s;
    const int64_t G = (int64_t)idx.G;
    ReadResult res{-1, -1, 0, kNotFound};
    st.reads++;
    if (m < s) {
        st.cls[kNotFound]++;
        return res;
    }
    std::vector<uint8_t> R(m), Rc(m);
    for (int i = 0; i < m; ++i) R[i] = (uint8_t)code_of(ascii[i]);
    for (int i = 0; i < m; ++i) Rc[i] = (uint8_t)(3 - R[m - 1 - i]);

    int n = P.n_seeds > 0 ? P.n_seeds : m / s;
    std::vector<int> offs;
    std::vector<uint8_t> pass0;
    seed_offsets(m, s, n, offs, pass0);
    n = (int)offs.size();

    struct Cand {
        int votes = 0;
        bool scored = false;
    };
    std::map<uint64_t, Cand> cand;  // key = 2p + strand, ascending
    struct Hit {
        uint64_t key;
        int d;
    };
    std::vector<Hit> hits;
    int d_best = kInf, d_second = kInf, best = -1, t = 0;
    bool any_nonpopular = false;
    const int d_max = P.d_max, c = P.c;

    // R9: seed g of the order above is looked up at offsets o, o+1, ..., o+stride-1
    // (those that fit in the read), so that one of them meets an indexed position
    // whatever the alignment; with stride 1 a probe is a seed.
    const int stride = idx.stride;
    std::vector<int> probe_off, probe_group;
    for (int g = 0; g < n; ++g)
        for (int j = 0; j < stride && offs[g] + j + s <= m; ++j) {
            probe_off.push_back(offs[g] + j);
            probe_group.push_back(g);
        }
    const int np = (int)probe_off.size();
    // probe lookups: the two position lists of each probe
    std::vector<std::vector<int64_t>> fwd_p(np), rc_p(np);
    std::vector<uint8_t> popular(np, 0);
    for (int i = 0; i < np; ++i) {
        const int o = probe_off[i];
        std::vector<uint8_t> S(R.begin() + o, R.begin() + o + s);
        std::vector<uint8_t> Src(s);
        for (int j = 0; j < s; ++j) Src[j] = (uint8_t)(3 - S[s - 1 - j]);
        uint64_t kS = kmer_value(S.data(), s), kR = kmer_value(Src.data(), s);
        auto a = idx.range(kS), b = idx.range(kR);
        uint64_t count = (a.second - a.first) + (b.second - b.first);
        st.seeds_looked_up++;
        if (count > (uint64_t)P.h_max) {
            popular[i] = 1;
            st.seeds_popular++;
            continue;
        }
        for (size_t q = a.first; q < a.second; ++q) {
            int64_t p = (int64_t)idx.entries[q].second - o;
            if (p >= 0 && p < G) fwd_p[i].push_back(p);
        }
        for (size_t q = b.first; q < b.second; ++q) {
            int64_t p = (int64_t)idx.entries[q].second - (m - o - s);
            if (p >= 0 && p < G) rc_p[i].push_back(p);
        }
    }

    auto distance = [&](uint64_t key, int L) -> int {
        const int64_t p = (int64_t)(key >> 1);
        const uint8_t* X = (key & 1) ? Rc.data() : R.data();
        int64_t avail = G - p;
        int64_t want = (int64_t)m + (L > 0 ? L : 0);
        int tn = (int)std::min(avail, want);
        return ed_lv(X, m, idx.genome.data() + p, tn, L);
    };

    // mode 1: speculate every candidate at L0
    std::map<uint64_t, int> d0;
    const int L0 = d_max + c - 1;
    if (mode == 1) {
        for (int i = 0; i < np; ++i) {
            for (int64_t p : fwd_p[i]) d0.emplace(2 * (uint64_t)p, 0);
            for (int64_t p : rc_p[i]) d0.emplace(2 * (uint64_t)p + 1, 0);
        }
        for (auto& kv : d0) kv.second = distance(kv.first, L0);
    }

    uint64_t calls_this_read = 0;
    auto bucket = [](uint64_t key) { return ((key >> 1) >> 5) * 2 + (key & 1); };
    auto limit = [&]() {
        if (d_best > d_max) return d_max + c - 1;
        if (d_second >= d_best + c) return d_best + c - 1;
        return d_best - 1;
    };
    auto pick = [&](uint64_t& out) {
        int bv = -1;
        for (auto& kv : cand) {
            if (!kv.second.scored && kv.second.votes > bv) {
                bv = kv.second.votes;
                out = kv.first;
            }
        }
        return bv >= 0;
    };
    auto score = [&](uint64_t key) {
        const int L = limit();
        int d;
        if (mode == 1) {
            int v = d0.at(key);
            d = (L >= 0 && v >= 0 && v <= L) ? v : -1;
        } else {
            d = distance(key, L);
        }
        st.ed_calls++;
        if (d < 0) st.ed_over++;
        if (calls_this_read > 0) {
            st.ed_calls_after_first++;
            if (d < 0) st.ed_over_after_first++;
        }
        calls_this_read++;
        cand[key].scored = true;
        if (d >= 0) {
            hits.push_back({key, d});
            d_best = kInf;
            best = -1;
            for (int j = 0; j < (int)hits.size(); ++j)
                if (hits[j].d < d_best) {
                    d_best = hits[j].d;
                    best = j;
                }
            d_second = kInf;
            const uint64_t bb = bucket(hits[best].key);
            for (const Hit& h : hits)
                if (bucket(h.key) != bb) d_second = std::min(d_second, h.d);
        }
    };
    auto finish_multiple = [&]() {
        res.cls = kMultiple;
        if (best >= 0 && d_best <= d_max) {
            res.location = (int64_t)(hits[best].key >> 1);
            res.strand = (uint8_t)(hits[best].key & 1);
            res.edit_distance = d_best;
        }
    };

    // R8: with first_seeds = k > 1 the first k non-popular seeds (all of them when
    // there are fewer) vote before anything is scored; afterwards one candidate per
    // seed as in Algorithm 1.  Before the first score no exit test can pass.
    // A seed counts as non-popular when one of its probes is (its votes are those
    // of its non-popular probes) and as tested for the Baeza-Yates bound (t) only
    // when it is from the unshifted pass and none of its probes was popular.
    std::vector<uint8_t> any_np(n, 0), all_np(n, 1);
    for (int i = 0; i < np; ++i) {
        if (popular[i]) all_np[probe_group[i]] = 0;
        else any_np[probe_group[i]] = 1;
    }
    int last_nonpopular = -1;
    for (int g = 0; g < n; ++g)
        if (any_np[g]) last_nonpopular = g;
    int voted = 0;
    bool returned = false;
    int pi = 0;  // first probe of seed g
    for (int g = 0; g < n && !returned; ++g) {
        const int p0 = pi;
        while (pi < np && probe_group[pi] == g) ++pi;
        if (!any_np[g]) continue;
        any_nonpopular = true;
        for (int i = p0; i < pi; ++i) {
            if (popular[i]) continue;
            for (int64_t p : fwd_p[i]) cand[2 * (uint64_t)p].votes++;
            for (int64_t p : rc_p[i]) cand[2 * (uint64_t)p + 1].votes++;
        }
        if (pass0[g] && all_np[g]) t++;
        ++voted;
        if (voted < P.first_seeds && g < last_nonpopular) continue;
        uint64_t k;
        if (pick(k)) score(k);
        if (d_best < c && d_second < d_best + c) {
            finish_multiple();
            returned = true;
            break;
        }
        if (t >= d_best + c) {
            while (pick(k)) score(k);
            break;
        }
    }
    st.candidates += cand.size();
    if (!hits.empty()) {
        st.reads_with_hit++;
        if (best == 0) st.first_scored_is_best++;
    }
    if (!returned) {
        bool all_popular = (np >= 1) && !any_nonpopular;
        if (d_best <= d_max && d_second >= d_best + c) {
            res.cls = kSingle;
            res.location = (int64_t)(hits[best].key >> 1);
            res.strand = (uint8_t)(hits[best].key & 1);
            res.edit_distance = d_best;
        } else if (d_best <= d_max || all_popular) {
            finish_multiple();
        } else {
            res.cls = kNotFound;
        }
    }
    st.cls[res.cls]++;
    return res;
}

}  // namespace

extern "C" {

struct or_result {
    int64_t location;
    int32_t edit_distance;
    uint8_t strand;
    uint8_t cls;
    uint8_t pad[2];
};

struct or_stats {
    uint64_t reads, seeds_looked_up, seeds_popular, ed_calls, ed_over, ed_calls_after_first,
        ed_over_after_first, reads_with_hit, first_scored_is_best, candidates, n_not_found,
        n_single, n_multiple;
};

// Build the oracle index over genome_ascii[0..G).  When filter != NULL (nfilter
// sorted s-mer values, first base most significant), only entries whose s-mer
// is in the filter are kept.  Returns NULL and sets *err on bad input.
void* or_index_build(const uint8_t* genome_ascii, uint64_t G, int s, int stride,
                     const uint64_t* filter, uint64_t nfilter, int* err) {
    if (err) *err = 0;
    if (!genome_ascii || s < 1 || s > 32 || G < (uint64_t)s || stride < 1) {
        if (err) *err = 1;
        return nullptr;
    }
    OracleIndex* idx = new OracleIndex();
    idx->s = s;
    idx->stride = stride;
    idx->G = G;
    idx->genome.resize(G);
    for (uint64_t i = 0; i < G; ++i) {
        int c = code_of(genome_ascii[i]);
        if (c < 0) {
            delete idx;
            if (err) *err = 2;
            return nullptr;
        }
        idx->genome[i] = (uint8_t)c;
    }
    const uint64_t npos = G - s + 1;
    const uint64_t mask = (s == 32) ? ~0ull : ((1ull << (2 * s)) - 1);
    std::vector<uint64_t> filt;
    if (filter) {
        filt.assign(filter, filter + nfilter);
        std::sort(filt.begin(), filt.end());
        idx->filtered = true;
    } else {
        idx->entries.reserve(npos);
    }
    if (!filter) {
        uint64_t v = kmer_value(idx->genome.data(), s);
        for (uint64_t l = 0; l < npos; ++l) {
            if (l > 0) v = ((v << 2) | idx->genome[l + s - 1]) & mask;
            if (l % (uint64_t)stride == 0) idx->entries.emplace_back(v, (uint32_t)l);
        }
    } else {
        // Restricted build: a bitmap of hashed filter keys screens each window
        // before the exact binary search, and position ranges are scanned by
        // several threads; the kept entries are exactly those of the full build
        // whose s-mer is in the filter.
        const int hb = 27;
        std::vector<uint64_t> bits((1ull << hb) / 64, 0);
        auto h = [&](uint64_t k) { return (k * 0x9E3779B97F4A7C15ull) >> (64 - hb); };
        for (uint64_t k : filt) bits[h(k) >> 6] |= 1ull << (h(k) & 63);
        int nt = (int)std::thread::hardware_concurrency();
        if (nt < 1) nt = 1;
        if (nt > 64) nt = 64;
        std::vector<std::vector<std::pair<uint64_t, uint32_t>>> part(nt);
        auto scan = [&](int t) {
            const uint64_t l0 = npos * t / nt, l1 = npos * (t + 1) / nt;
            if (l0 >= l1) return;
            uint64_t v = kmer_value(idx->genome.data() + l0, s);
            for (uint64_t l = l0; l < l1; ++l) {
                if (l > l0) v = ((v << 2) | idx->genome[l + s - 1]) & mask;
                if (l % (uint64_t)stride != 0) continue;
                const uint64_t hv = h(v);
                if (!(bits[hv >> 6] >> (hv & 63) & 1)) continue;
                if (std::binary_search(filt.begin(), filt.end(), v))
                    part[t].emplace_back(v, (uint32_t)l);
            }
        };
        std::vector<std::thread> th;
        for (int t = 0; t < nt; ++t) th.emplace_back(scan, t);
        for (auto& x : th) x.join();
        for (auto& pv : part) idx->entries.insert(idx->entries.end(), pv.begin(), pv.end());
    }
    std::sort(idx->entries.begin(), idx->entries.end());
    return idx;
}

void or_index_free(void* h) { delete static_cast<OracleIndex*>(h); }

uint64_t or_index_entries(void* h) { return static_cast<OracleIndex*>(h)->entries.size(); }

// Forward occurrences of one s-mer given as ASCII; writes up to cap positions.
uint64_t or_index_occurrences(void* h, const uint8_t* smer_ascii, uint32_t* out, uint64_t cap) {
    const OracleIndex* idx = static_cast<OracleIndex*>(h);
    std::vector<uint8_t> c(idx->s);
    for (int j = 0; j < idx->s; ++j) {
        int x = code_of(smer_ascii[j]);
        if (x < 0) return 0;
        c[j] = (uint8_t)x;
    }
    auto r = idx->range(kmer_value(c.data(), idx->s));
    uint64_t n = r.second - r.first;
    for (uint64_t q = 0; q < n && q < cap; ++q) out[q] = idx->entries[r.first + q].second;
    return n;
}

int or_seed_offsets(int m, int s, int n, int32_t* offs, uint8_t* pass0, int cap) {
    std::vector<int> o;
    std::vector<uint8_t> p;
    seed_offsets(m, s, n, o, p);
    for (int i = 0; i < (int)o.size() && i < cap; ++i) {
        offs[i] = o[i];
        pass0[i] = p[i];
    }
    return (int)o.size();
}

static bool to_codes(const uint8_t* a, int n, std::vector<uint8_t>& out) {
    out.resize(n);
    for (int i = 0; i < n; ++i) {
        int c = code_of(a[i]);
        if (c < 0) return false;
        out[i] = (uint8_t)c;
    }
    return true;
}

// Bounded distance (farthest reach per diagonal); -1 = over the limit, -2 = bad base.
int or_ed_lv(const uint8_t* x_ascii, int m, const uint8_t* t_ascii, int n, int L) {
    std::vector<uint8_t> x, t;
    if (!to_codes(x_ascii, m, x) || !to_codes(t_ascii, n, t)) return -2;
    return ed_lv(x.data(), m, t.data(), n, L);
}

// Textbook table, anchored start and free end in the text; -2 = bad base.
int or_ed_dp(const uint8_t* x_ascii, int m, const uint8_t* t_ascii, int n) {
    std::vector<uint8_t> x, t;
    if (!to_codes(x_ascii, m, x) || !to_codes(t_ascii, n, t)) return -2;
    return ed_dp(x.data(), m, t.data(), n);
}

// Many (X, T, L) triples at once: out_lv[i] = bounded distance (or -1), and
// out_dp[i] = the full-table distance when out_dp != NULL.  -2 marks a bad base.
void or_ed_pairs(const uint8_t* xs, const uint64_t* xoff, const uint8_t* ts, const uint64_t* toff,
                 const int32_t* L, uint64_t n, int32_t* out_lv, int32_t* out_dp) {
    std::vector<uint8_t> x, t;
    for (uint64_t i = 0; i < n; ++i) {
        int m = (int)(xoff[i + 1] - xoff[i]), tn = (int)(toff[i + 1] - toff[i]);
        if (!to_codes(xs + xoff[i], m, x) || !to_codes(ts + toff[i], tn, t)) {
            out_lv[i] = -2;
            if (out_dp) out_dp[i] = -2;
            continue;
        }
        out_lv[i] = ed_lv(x.data(), m, t.data(), tn, L[i]);
        if (out_dp) out_dp[i] = ed_dp(x.data(), m, t.data(), tn);
    }
}

// The s-mer values of every seed of every read (every probe of it, R9, for a
// strided index) and of their reverse complements (the lookups Algorithm 1
// makes), for a filtered index.  Returns
// the number written (<= cap) or the number needed when out == NULL.
uint64_t or_read_seed_kmers(const uint8_t* reads, const uint64_t* offsets, uint64_t nreads, int s,
                            int n_seeds, int stride, uint64_t* out, uint64_t cap) {
    uint64_t k = 0;
    std::vector<int> offs, probes;
    std::vector<uint8_t> pass0, S(s), Src(s);
    if (stride < 1) stride = 1;
    for (uint64_t r = 0; r < nreads; ++r) {
        const uint8_t* a = reads + offsets[r];
        int m = (int)(offsets[r + 1] - offsets[r]);
        int n = n_seeds > 0 ? n_seeds : (s > 0 ? m / s : 0);
        seed_offsets(m, s, n, offs, pass0);
        probes.clear();  // R9: each seed's probes
        for (int o0 : offs)
            for (int j = 0; j < stride && o0 + j + s <= m; ++j) probes.push_back(o0 + j);
        for (int o : probes) {
            bool ok = true;
            for (int j = 0; j < s; ++j) {
                int c = code_of(a[o + j]);
                if (c < 0) ok = false;
                S[j] = (uint8_t)(c < 0 ? 0 : c);
            }
            if (!ok) continue;
            for (int j = 0; j < s; ++j) Src[j] = (uint8_t)(3 - S[s - 1 - j]);
            if (out && k < cap) out[k] = kmer_value(S.data(), s);
            k++;
            if (out && k < cap) out[k] = kmer_value(Src.data(), s);
            k++;
        }
    }
    return k;
}

// Align reads[offsets[r]..offsets[r+1]) for r < n.  mode 0 literal, 1
// speculate-and-replay.  dmax_per_read overrides d_max per read when non-NULL.
// first_seeds <= 1 is Algorithm 1, k > 1 its seeds-first variant (R8).
// threads <= 0 means one.  Returns 0, or 1 on bad input (non-ACGT base).
int or_align(void* h, const uint8_t* reads, const uint64_t* offsets, uint64_t n, int d_max,
             int h_max, int c, int n_seeds, int first_seeds, const int32_t* dmax_per_read,
             int mode, int threads, or_result* out, or_stats* stats) {
    const OracleIndex* idx = static_cast<OracleIndex*>(h);
    if (!idx || !reads || !offsets || !out) return 1;
    for (uint64_t r = 0; r < n; ++r)
        for (uint64_t q = offsets[r]; q < offsets[r + 1]; ++q)
            if (code_of(reads[q]) < 0) return 1;
    if (threads < 1) threads = 1;
    if ((uint64_t)threads > n) threads = n ? (int)n : 1;
    std::vector<Stats> st(threads);
    auto work = [&](int tix) {
        uint64_t r0 = n * tix / threads, r1 = n * (tix + 1) / threads;
        for (uint64_t r = r0; r < r1; ++r) {
            Params P{dmax_per_read ? dmax_per_read[r] : d_max, h_max, c, n_seeds, first_seeds};
            ReadResult rr = align_one(*idx, reads + offsets[r], (int)(offsets[r + 1] - offsets[r]),
                                      P, mode, st[tix]);
            out[r].location = rr.location;
            out[r].edit_distance = rr.edit_distance;
            out[r].strand = rr.strand;
            out[r].cls = rr.cls;
            out[r].pad[0] = out[r].pad[1] = 0;
        }
    };
    if (threads == 1) {
        work(0);
    } else {
        std::vector<std::thread> th;
        for (int t = 0; t < threads; ++t) th.emplace_back(work, t);
        for (auto& x : th) x.join();
    }
    if (stats) {
        Stats all;
        for (auto& x : st) all.add(x);
        stats->reads = all.reads;
        stats->seeds_looked_up = all.seeds_looked_up;
        stats->seeds_popular = all.seeds_popular;
        stats->ed_calls = all.ed_calls;
        stats->ed_over = all.ed_over;
        stats->ed_calls_after_first = all.ed_calls_after_first;
        stats->ed_over_after_first = all.ed_over_after_first;
        stats->reads_with_hit = all.reads_with_hit;
        stats->first_scored_is_best = all.first_scored_is_best;
        stats->candidates = all.candidates;
        stats->n_not_found = all.cls[kNotFound];
        stats->n_single = all.cls[kSingle];
        stats->n_multiple = all.cls[kMultiple];
    }
    return 0;
}

}  // extern "C"
