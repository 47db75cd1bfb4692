/*
 * synth.c — seeded synthetic inputs for the SNAP alignment workloads.
 *
 * This module only makes inputs: a reference genome (uniform ACGT plus
 * near-duplicate repeat families), simulated reads with a known origin, read
 * length mixes and Poisson request arrivals.  It holds none of the alignment
 * method's arithmetic (no seeds, no index, no edit distance), so the oracle and
 * the CUDA path can both consume its output without sharing any logic.
 *
 * The paper evaluates on simulated reads with a known true location (Results
 * section, "simulated reads"), on hg19/wgsim and on NA12878; none of those are
 * available here, so these generators stand in for them.  The repeat-family
 * model mimics the near-duplicate clusters described in the "Observations"
 * subsection of "Ongoing Work" (hundreds of similar strings differing in a few
 * bases).
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018) seeded through
 * splitmix64 (Steele, Lea & Flood, 2014), both restated from their published
 * definitions.  Every read draws from its own stream keyed by (seed, index),
 * so reads can be generated in parallel, or any sub-range alone, with
 * identical results.  Integer arithmetic is used wherever a value decides a
 * base; log/exp only shape lengths and gaps.
 *
 * Encoding of the output: ASCII 'A','C','G','T' (uppercase), one byte per base.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s[4]; } srng;

static uint64_t splitmix64_next(uint64_t* x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static void srng_seed(srng* r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64_next(&x);
}

static inline uint64_t srng_next(srng* r) {
    uint64_t* s = r->s;
    const uint64_t result = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

/* Stream for item `idx` of a family of streams keyed by `seed`. */
static void srng_seed2(srng* r, uint64_t seed, uint64_t idx) {
    uint64_t x = seed ^ 0x5851F42D4C957F2Dull;
    uint64_t a = splitmix64_next(&x);
    uint64_t y = a ^ (idx * 0xD1B54A32D192ED03ull + 0x632BE59BD9B4E019ull);
    srng_seed(r, splitmix64_next(&y));
}

/* uniform in [0,1) with 53 random bits */
static inline double srng_u01(srng* r) { return (double)(srng_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* uniform integer in [lo, hi] (hi - lo < 2^32), by the high half of a 64x32 product */
static inline uint64_t srng_uint(srng* r, uint64_t lo, uint64_t hi) {
    uint64_t span = hi - lo + 1;
    uint64_t x = srng_next(r) >> 32;
    return lo + ((x * span) >> 32);
}

/* uniform integer in [0, n) for n up to 2^63, by 128-bit multiply-high */
static inline uint64_t srng_below(srng* r, uint64_t n) {
    return (uint64_t)(((unsigned __int128)srng_next(r) * n) >> 64);
}

/* number of failures before the first success of Bernoulli(p) trials */
static inline uint64_t srng_geom(srng* r, double p) {
    if (p <= 0.0) return UINT64_MAX;
    if (p >= 1.0) return 0;
    double u = 1.0 - srng_u01(r); /* (0,1] */
    double g = floor(log(u) / log1p(-p));
    if (g > 1e18) return UINT64_MAX;
    return (uint64_t)g;
}

static const uint8_t kBase[4] = {'A', 'C', 'G', 'T'};

static inline uint8_t comp_ascii(uint8_t b) {
    switch (b) {
        case 'A': return 'T';
        case 'C': return 'G';
        case 'G': return 'C';
        default: return 'A';
    }
}

/* a base different from b, uniformly among the other three */
static inline uint8_t other_base(srng* r, uint8_t b) {
    int code = (b == 'A') ? 0 : (b == 'C') ? 1 : (b == 'G') ? 2 : 3;
    int k = (int)srng_uint(r, 1, 3);
    return kBase[(code + k) & 3];
}

/* ------------------------------------------------------------------------ */
/* genome                                                                     */
/* ------------------------------------------------------------------------ */

#define CHUNK_BASES (1u << 20)

typedef struct {
    uint8_t* out;
    uint64_t G, seed;
    uint64_t c0, c1; /* chunk range */
} genome_job;

static void* genome_worker(void* arg) {
    genome_job* j = (genome_job*)arg;
    for (uint64_t c = j->c0; c < j->c1; ++c) {
        srng r;
        srng_seed2(&r, j->seed, c);
        uint64_t b0 = c * (uint64_t)CHUNK_BASES;
        uint64_t b1 = b0 + CHUNK_BASES;
        if (b1 > j->G) b1 = j->G;
        uint64_t x = 0;
        for (uint64_t i = b0; i < b1; ++i) {
            if (((i - b0) & 31) == 0) x = srng_next(&r);
            j->out[i] = kBase[x >> 62];
            x <<= 2;
        }
    }
    return NULL;
}

/*
 * Uniform i.i.d. ACGT genome of length G (stream `seed_genome`, chunked so it
 * can be filled by `threads` threads), then repeat families until at least
 * repeat_frac*G bases are covered by some copy (stream `seed_repeats`):
 *   unit length U ~ U[unit_lo, unit_hi], copies K ~ U[copies_lo, copies_hi],
 *   a random source unit, each copy placed at a uniform position with i.i.d.
 *   substitutions at rate `divergence`; later copies overwrite earlier ones.
 * Returns the number of covered bases in *covered_out.
 */
int synth_genome(uint8_t* out, uint64_t G, double repeat_frac, uint64_t seed_genome,
                 uint64_t seed_repeats, uint32_t unit_lo, uint32_t unit_hi, uint32_t copies_lo,
                 uint32_t copies_hi, double divergence, int threads, uint64_t* covered_out) {
    if (!out || G == 0) return 1;
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    uint64_t nchunks = (G + CHUNK_BASES - 1) / CHUNK_BASES;
    pthread_t tid[256];
    genome_job jobs[256];
    int nt = threads;
    if ((uint64_t)nt > nchunks) nt = (int)nchunks;
    for (int t = 0; t < nt; ++t) {
        jobs[t].out = out;
        jobs[t].G = G;
        jobs[t].seed = seed_genome;
        jobs[t].c0 = nchunks * t / nt;
        jobs[t].c1 = nchunks * (t + 1) / nt;
        pthread_create(&tid[t], NULL, genome_worker, &jobs[t]);
    }
    for (int t = 0; t < nt; ++t) pthread_join(tid[t], NULL);

    uint64_t covered = 0;
    uint64_t target = (uint64_t)(repeat_frac * (double)G);
    if (repeat_frac > 0.0 && target > 0) {
        if (unit_lo < 1) unit_lo = 1;
        if (unit_hi < unit_lo) unit_hi = unit_lo;
        if (copies_hi < copies_lo) copies_hi = copies_lo;
        uint64_t* bitmap = (uint64_t*)calloc((G + 63) / 64, sizeof(uint64_t));
        uint8_t* unit = (uint8_t*)malloc(unit_hi);
        if (!bitmap || !unit) {
            free(bitmap);
            free(unit);
            return 2;
        }
        srng r;
        srng_seed(&r, seed_repeats);
        while (covered < target) {
            uint64_t U = srng_uint(&r, unit_lo, unit_hi);
            if (U > G) U = G;
            uint64_t K = srng_uint(&r, copies_lo, copies_hi);
            for (uint64_t j = 0; j < U; ++j) unit[j] = kBase[srng_next(&r) >> 62];
            for (uint64_t c = 0; c < K && covered < target; ++c) {
                uint64_t pos = srng_below(&r, G - U + 1);
                memcpy(out + pos, unit, U);
                /* substitutions by geometric skipping */
                uint64_t j = srng_geom(&r, divergence);
                while (j < U) {
                    out[pos + j] = other_base(&r, unit[j]);
                    uint64_t g = srng_geom(&r, divergence);
                    if (g >= U) break;
                    j += g + 1;
                }
                for (uint64_t q = pos; q < pos + U; ++q) {
                    uint64_t w = q >> 6, bit = 1ull << (q & 63);
                    if (!(bitmap[w] & bit)) {
                        bitmap[w] |= bit;
                        ++covered;
                    }
                }
            }
        }
        free(bitmap);
        free(unit);
    }
    if (covered_out) *covered_out = covered;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* read lengths and request arrivals                                          */
/* ------------------------------------------------------------------------ */

/* floor(lo * (hi/lo)^u), clamped to [lo, hi] */
static uint32_t log_uniform_len(srng* r, uint32_t lo, uint32_t hi) {
    if (hi <= lo) return lo;
    double u = srng_u01(r);
    double v = exp(log((double)lo) + u * (log((double)hi + 1.0) - log((double)lo)));
    uint64_t m = (uint64_t)floor(v);
    if (m < lo) m = lo;
    if (m > hi) m = hi;
    return (uint32_t)m;
}

/*
 * mode 0: every length = m_fixed
 * mode 1: log-uniform in [lo, hi]
 * mode 2: with probability frac_fixed the length is m_fixed, else log-uniform in [lo, hi]
 */
int synth_read_lengths(uint32_t* lens, uint64_t n, int mode, uint32_t m_fixed, uint32_t lo,
                       uint32_t hi, double frac_fixed, uint64_t seed) {
    if (!lens) return 1;
    srng r;
    srng_seed(&r, seed);
    for (uint64_t i = 0; i < n; ++i) {
        if (mode == 0) {
            lens[i] = m_fixed;
        } else if (mode == 1) {
            lens[i] = log_uniform_len(&r, lo, hi);
        } else {
            double u = srng_u01(&r);
            uint32_t l = log_uniform_len(&r, lo, hi);
            lens[i] = (u < frac_fixed) ? m_fixed : l;
        }
    }
    return 0;
}

/* Poisson arrivals at `rate` per second and log-uniform request sizes in [lo, hi]. */
int synth_arrivals(double* times, uint32_t* sizes, uint64_t n_req, double rate, uint32_t lo,
                   uint32_t hi, uint64_t seed_arrivals, uint64_t seed_sizes) {
    if (!times || !sizes || rate <= 0.0) return 1;
    srng ra, rs;
    srng_seed(&ra, seed_arrivals);
    srng_seed(&rs, seed_sizes);
    double t = 0.0;
    for (uint64_t i = 0; i < n_req; ++i) {
        double u = 1.0 - srng_u01(&ra);
        t += -log(u) / rate;
        times[i] = t;
        sizes[i] = log_uniform_len(&rs, lo, hi);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* reads                                                                      */
/* ------------------------------------------------------------------------ */

typedef struct {
    const uint8_t* genome;
    uint64_t G;
    const uint32_t* lens;
    const uint64_t* offsets;
    uint64_t first_index; /* global index of read 0 of this call */
    uint64_t r0, r1;
    double sub_rate, indel_rate;
    uint32_t indel_lo, indel_hi;
    uint64_t seed;
    uint8_t* out;
    int64_t* t_origin;
    uint8_t* t_strand;
    uint32_t* t_edits;
} reads_job;

static void make_one_read(const reads_job* j, uint64_t i) {
    srng r;
    srng_seed2(&r, j->seed, j->first_index + i);
    uint64_t m = j->lens[i];
    uint8_t* dst = j->out + j->offsets[i];
    uint64_t span = (uint64_t)ceil(1.5 * (double)m);
    uint64_t hi = (j->G > span) ? (j->G - span) : 0;
    uint64_t origin = srng_below(&r, hi + 1);
    uint64_t g = origin, k = 0;
    uint32_t edits = 0;
    uint64_t indel_cd = srng_geom(&r, j->indel_rate);
    uint64_t sub_cd = srng_geom(&r, j->sub_rate);
    while (k < m) {
        if (indel_cd == 0) {
            uint64_t L = srng_uint(&r, j->indel_lo, j->indel_hi);
            ++edits;
            if (srng_next(&r) >> 63) {
                for (uint64_t q = 0; q < L && k < m; ++q) dst[k++] = kBase[srng_next(&r) >> 62];
            } else {
                g += L;
            }
            indel_cd = srng_geom(&r, j->indel_rate);
            if (k >= m) break;
        } else if (indel_cd != UINT64_MAX) {
            --indel_cd;
        }
        uint8_t b = (g < j->G) ? j->genome[g] : kBase[srng_next(&r) >> 62];
        ++g;
        if (sub_cd == 0) {
            b = other_base(&r, b);
            ++edits;
            sub_cd = srng_geom(&r, j->sub_rate);
        } else if (sub_cd != UINT64_MAX) {
            --sub_cd;
        }
        dst[k++] = b;
    }
    uint8_t strand = (uint8_t)(srng_next(&r) >> 63);
    if (strand && m > 0) {
        uint64_t a = 0, b = m - 1;
        while (a < b) {
            uint8_t x = comp_ascii(dst[a]), y = comp_ascii(dst[b]);
            dst[a++] = y;
            dst[b--] = x;
        }
        if (a == b) dst[a] = comp_ascii(dst[a]);
    }
    if (j->t_origin) j->t_origin[i] = (int64_t)origin;
    if (j->t_strand) j->t_strand[i] = strand;
    if (j->t_edits) j->t_edits[i] = edits;
}

static void* reads_worker(void* arg) {
    reads_job* j = (reads_job*)arg;
    for (uint64_t i = j->r0; i < j->r1; ++i) make_one_read(j, i);
    return NULL;
}

/*
 * Simulated reads.  For read i (stream (seed, first_index + i)): origin uniform
 * in [0, G - ceil(1.5 m)]; walk the reference from the origin; before each
 * emitted base an indel event happens with probability indel_rate (length
 * uniform in [indel_lo, indel_hi], insertion of random bases or deletion of
 * reference bases, 50/50); each emitted reference base is replaced by one of
 * the other three with probability sub_rate; stop at m bases; finally the read
 * is reverse-complemented with probability 1/2.  Truth is (origin, strand,
 * number of edit events).  offsets[] (n+1 entries) is filled from lens[] when
 * fill_offsets != 0, else taken as given.
 */
int synth_reads(const uint8_t* genome, uint64_t G, const uint32_t* lens, uint64_t n,
                uint64_t first_index, double sub_rate, double indel_rate, uint32_t indel_lo,
                uint32_t indel_hi, uint64_t seed, uint8_t* out, uint64_t* offsets, int fill_offsets,
                int64_t* t_origin, uint8_t* t_strand, uint32_t* t_edits, int threads) {
    if (!genome || !lens || !out || !offsets || G == 0) return 1;
    if (indel_hi < indel_lo) indel_hi = indel_lo;
    if (fill_offsets) {
        offsets[0] = 0;
        for (uint64_t i = 0; i < n; ++i) offsets[i + 1] = offsets[i] + lens[i];
    }
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    int nt = threads;
    if ((uint64_t)nt > n) nt = n ? (int)n : 1;
    pthread_t tid[256];
    reads_job jobs[256];
    for (int t = 0; t < nt; ++t) {
        reads_job* j = &jobs[t];
        j->genome = genome;
        j->G = G;
        j->lens = lens;
        j->offsets = offsets;
        j->first_index = first_index;
        j->r0 = n * t / nt;
        j->r1 = n * (t + 1) / nt;
        j->sub_rate = sub_rate;
        j->indel_rate = indel_rate;
        j->indel_lo = indel_lo;
        j->indel_hi = indel_hi;
        j->seed = seed;
        j->out = out;
        j->t_origin = t_origin;
        j->t_strand = t_strand;
        j->t_edits = t_edits;
        pthread_create(&tid[t], NULL, reads_worker, j);
    }
    for (int t = 0; t < nt; ++t) pthread_join(tid[t], NULL);
    return 0;
}

/* raw stream access, for tests of the generator itself */
uint64_t synth_rng_first(uint64_t seed, uint64_t* out, uint64_t n) {
    srng r;
    srng_seed(&r, seed);
    for (uint64_t i = 0; i < n; ++i) out[i] = srng_next(&r);
    return n;
}
