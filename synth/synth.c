/*
 * Seeded synthetic inputs for the seeding stage: reference genomes and reads.
 *
 * This module holds no arithmetic of the method (no suffix array, BWT,
 * occurrence counts, SMEMs or locate).  It only draws random sequences with
 * the shapes of the workloads the paper evaluates on (2x150 bp short-read WGS
 * and mixed-length reads, Section 3.1), which are not available here.  Both
 * the CPU oracle and the GPU path read what it writes.
 *
 * Randomness: every independent unit (a chunk of reference, a repeat element,
 * a read) gets its own xoshiro256** stream seeded through splitmix64 from
 * (seed, stream id), so the output does not depend on thread count.
 *   splitmix64: G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom
 *   number generators", OOPSLA 2014.
 *   xoshiro256**: D. Blackman, S. Vigna, "Scrambled linear pseudorandom number
 *   generators", ACM TOMS 2021.
 *
 * Base codes: 0=A 1=C 2=G 3=T 4=N.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t sm64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static void rng_init(rng_t *r, uint64_t seed, uint64_t stream) {
    uint64_t x = seed ^ (stream * 0xD1B54A32D192ED03ULL);
    for (int i = 0; i < 4; ++i) r->s[i] = sm64_next(&x);
}

static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t rng_u64(rng_t *r) {
    uint64_t *s = r->s;
    uint64_t res = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl(s[3], 45);
    return res;
}

/* uniform double in [0,1) */
static inline double rng_unif(rng_t *r) { return (rng_u64(r) >> 11) * (1.0 / 9007199254740992.0); }
/* uniform integer in [0, m) (m > 0), by multiply-shift */
static inline uint64_t rng_below(rng_t *r, uint64_t m) {
    return (uint64_t)(((__uint128_t)rng_u64(r) * m) >> 64);
}
/* uniform integer in [lo, hi] */
static inline uint64_t rng_range(rng_t *r, uint64_t lo, uint64_t hi) { return lo + rng_below(r, hi - lo + 1); }
static inline uint8_t rng_base(rng_t *r) { return (uint8_t)(rng_u64(r) >> 62); }
/* a base different from b (b in 0..3) */
static inline uint8_t rng_other(rng_t *r, uint8_t b) { return (uint8_t)((b + 1 + rng_below(r, 3)) & 3); }
/*
 * Only +,-,*,/ below (IEEE-exact on every platform; the library is built with
 * -ffp-contract=off), so x86 and Arm hosts draw identical inputs.
 */
/* approximately standard normal: Irwin-Hall sum of 12 uniforms minus 6 */
static double rng_normal(rng_t *r) {
    double s = 0;
    for (int i = 0; i < 12; ++i) s += rng_unif(r);
    return s - 6.0;
}
/* e^x by argument halving and a Taylor series */
static double det_exp(double x) {
    int h = 0;
    while (x > 0.5 || x < -0.5) { x *= 0.5; ++h; }
    double term = 1, sum = 1;
    for (int k = 1; k < 24; ++k) { term = term * x / k; sum += term; }
    while (h-- > 0) sum *= sum;
    return sum;
}
/* natural log of y > 0 by Newton iterations on det_exp */
static double det_log(double y) {
    double x = 0, t = y;
    while (t > 2) { t *= 0.5; x += 0.6931471805599453; }
    while (t < 0.5) { t *= 2; x -= 0.6931471805599453; }
    for (int i = 0; i < 40; ++i) x = x - 1.0 + y / det_exp(x);
    return x;
}

static inline uint8_t comp(uint8_t b) { return b < 4 ? (uint8_t)(3 - b) : b; }

/* copy src[0,len) into dst with i.i.d. substitutions at rate d (N kept) */
static void mutate_copy(rng_t *r, uint8_t *dst, const uint8_t *src, uint64_t len, double d) {
    for (uint64_t i = 0; i < len; ++i) {
        uint8_t b = src[i];
        if (b < 4 && d > 0 && rng_unif(r) < d) b = rng_other(r, b);
        dst[i] = b;
    }
}

#define CHUNK (1u << 20)

/*
 * Reference genome.  len bases; fractions of len covered by tandem arrays
 * (period 1-200, 2-500 copies, divergence 0-3%), segmental duplications
 * (1-50 kb, divergence 1-5%, half reverse-complemented, copied from elsewhere
 * in the sequence), satellite arrays (one 171 bp consensus, 20-500 monomers at
 * 2% divergence) and N runs (100-10,000 bp).  The rest is i.i.d. uniform.
 * Elements are placed at uniform positions and may overwrite one another.
 */
void synth_ref(uint8_t *out, uint64_t len, uint64_t seed, double f_tandem, double f_segdup,
               double f_sat, double f_n) {
    uint64_t nchunk = (len + CHUNK - 1) / CHUNK;
#pragma omp parallel for schedule(static)
    for (uint64_t c = 0; c < nchunk; ++c) {
        rng_t r; rng_init(&r, seed, c);
        uint64_t b = c * CHUNK, e = b + CHUNK < len ? b + CHUNK : len;
        for (uint64_t i = b; i < e; i += 32) {
            uint64_t w = rng_u64(&r);
            for (uint64_t k = i; k < e && k < i + 32; ++k, w >>= 2) out[k] = (uint8_t)(w & 3);
        }
    }
    if (len < 1000) return;
    uint64_t stream = 1ULL << 40;
    rng_t g; rng_init(&g, seed, stream++);
    /* tandem repeats */
    double budget = f_tandem * (double)len, done = 0;
    uint8_t unit[200];
    uint8_t *tmp = (uint8_t *)malloc(200 * 500 + 60000);
    while (done < budget) {
        uint64_t p = rng_range(&g, 1, 200), cp = rng_range(&g, 2, 500);
        double d = rng_unif(&g) * 0.03;
        uint64_t tot = p * cp;
        if (tot >= len / 2) continue;
        uint64_t pos = rng_below(&g, len - tot);
        rng_t e; rng_init(&e, seed, stream++);
        for (uint64_t i = 0; i < p; ++i) unit[i] = rng_base(&e);
        for (uint64_t c = 0; c < cp; ++c) mutate_copy(&e, out + pos + c * p, unit, p, d);
        done += (double)tot;
    }
    /* satellite arrays of one 171 bp consensus */
    uint8_t cons[171];
    { rng_t e; rng_init(&e, seed, stream++); for (int i = 0; i < 171; ++i) cons[i] = rng_base(&e); }
    budget = f_sat * (double)len; done = 0;
    while (done < budget) {
        uint64_t m = rng_range(&g, 20, 500), tot = m * 171;
        if (tot >= len / 2) { if (len < 2 * 171 * 20) break; continue; }
        uint64_t pos = rng_below(&g, len - tot);
        rng_t e; rng_init(&e, seed, stream++);
        for (uint64_t c = 0; c < m; ++c) mutate_copy(&e, out + pos + c * 171, cons, 171, 0.02);
        done += (double)tot;
    }
    /* segmental duplications */
    budget = f_segdup * (double)len; done = 0;
    while (done < budget) {
        uint64_t L = rng_range(&g, 1000, 50000);
        if (2 * L >= len) { if (len < 4000) break; continue; }
        uint64_t src = rng_below(&g, len - L), dst = rng_below(&g, len - L);
        double d = 0.01 + rng_unif(&g) * 0.04;
        int rc = (int)(rng_u64(&g) >> 63);
        rng_t e; rng_init(&e, seed, stream++);
        memcpy(tmp, out + src, L);
        if (rc) for (uint64_t i = 0; i < L / 2; ++i) {
            uint8_t a = comp(tmp[i]), b = comp(tmp[L - 1 - i]);
            tmp[i] = b; tmp[L - 1 - i] = a;
        }
        if (rc && (L & 1)) tmp[L / 2] = comp(tmp[L / 2]);
        mutate_copy(&e, out + dst, tmp, L, d);
        done += (double)L;
    }
    /* N runs */
    budget = f_n * (double)len; done = 0;
    while (done < budget) {
        uint64_t L = rng_range(&g, 100, 10000);
        if (2 * L >= len) break;
        uint64_t pos = rng_below(&g, len - L);
        memset(out + pos, 4, L);
        done += (double)L;
    }
    free(tmp);
}

/* Read set parameters. */
typedef struct {
    int mode;            /* 0 = single-end fixed length, 1 = paired-end, 2 = single-end log-uniform length */
    uint32_t read_len;   /* modes 0,1 */
    uint32_t len_lo, len_hi;   /* mode 2 */
    double sub_lo, sub_hi;     /* substitution rate ramps linearly from sub_lo (first base) to sub_hi (last) */
    double indel;        /* per-base indel rate, length 1-3, insertion/deletion 50/50 */
    double frag_mean, frag_sd;   /* mode 1 */
    int bisulfite;       /* mode 1: directional bisulfite conversion of the fragment */
    double bs_noncpg, bs_cpg;    /* conversion rates of C outside / inside CpG */
} synth_read_opts;

static uint32_t read_length(const synth_read_opts *o, uint64_t seed, uint64_t rid) {
    if (o->mode != 2) return o->read_len;
    rng_t r; rng_init(&r, seed ^ 0x4C454E47ULL, rid);
    double lo = det_log((double)o->len_lo), hi = det_log((double)o->len_hi);
    double L = det_exp(lo + (hi - lo) * rng_unif(&r));
    uint32_t l = (uint32_t)(L + 0.5);
    if (l < o->len_lo) l = o->len_lo;
    if (l > o->len_hi) l = o->len_hi;
    return l;
}

/* Lengths of all reads (a pair counts as two reads of read_len). */
uint64_t synth_read_lengths(const synth_read_opts *o, uint64_t seed, uint32_t n_reads, uint64_t *off) {
    off[0] = 0;
    for (uint32_t i = 0; i < n_reads; ++i) off[i + 1] = off[i] + read_length(o, seed, i);
    return off[n_reads];
}

/*
 * Emit one read of length L from the template tpl[0, tl) (already in read
 * orientation), applying position-dependent substitutions and indels.
 */
static void emit_read(rng_t *r, const synth_read_opts *o, const uint8_t *tpl, uint64_t tl,
                      uint8_t *dst, uint32_t L) {
    uint64_t t = 0;
    uint32_t x = 0;
    while (x < L) {
        if (o->indel > 0 && rng_unif(r) < o->indel) {
            uint32_t il = (uint32_t)rng_range(r, 1, 3);
            if (rng_u64(r) >> 63) {            /* insertion */
                for (uint32_t q = 0; q < il && x < L; ++q) dst[x++] = rng_base(r);
                continue;
            } else {                            /* deletion */
                t += il;
            }
        }
        uint8_t b = t < tl ? tpl[t] : rng_base(r);
        ++t;
        double p = o->sub_lo + (L > 1 ? (o->sub_hi - o->sub_lo) * (double)x / (double)(L - 1) : 0.0);
        if (b < 4 && p > 0 && rng_unif(r) < p) b = rng_other(r, b);
        dst[x++] = b;
    }
}

/*
 * Reads sampled from ref[0,ref_len) on both strands.  off must come from
 * synth_read_lengths.  For paired-end mode, reads 2i and 2i+1 are mates;
 * read 2 is the reverse complement of the fragment's far end.  origin (may be
 * NULL) receives the forward-strand start of each read's template and its
 * strand in bit 63.
 */
void synth_reads(const uint8_t *ref, uint64_t ref_len, const synth_read_opts *o, uint64_t seed,
                 uint32_t n_reads, const uint64_t *off, uint8_t *seq, uint64_t *origin) {
    uint32_t n_units = o->mode == 1 ? n_reads / 2 : n_reads;
#pragma omp parallel
    {
        uint64_t cap = 0;
        uint8_t *frag = NULL;
#pragma omp for schedule(dynamic, 256)
        for (uint32_t u = 0; u < n_units; ++u) {
            rng_t r; rng_init(&r, seed, (uint64_t)u + 7);
            if (o->mode == 1) {
                uint32_t L = o->read_len;
                double f = o->frag_mean + o->frag_sd * rng_normal(&r);
                uint64_t F = f < L ? L : (uint64_t)(f + 0.5);
                if (F + 16 > ref_len) F = ref_len > 16 + L ? ref_len - 16 : L;
                uint64_t need = F + 16;
                if (2 * need > cap) { free(frag); cap = 2 * need; frag = (uint8_t *)malloc(cap); }
                uint64_t start = rng_below(&r, ref_len - need + 1);
                int strand = (int)(rng_u64(&r) >> 63);
                for (uint64_t q = 0; q < need; ++q)
                    frag[q] = strand ? comp(ref[start + need - 1 - q]) : ref[start + q];
                if (o->bisulfite) {
                    for (uint64_t q = 0; q < need; ++q) if (frag[q] == 1) {
                        int cpg = q + 1 < need && frag[q + 1] == 2;
                        if (rng_unif(&r) < (cpg ? o->bs_cpg : o->bs_noncpg)) frag[q] = 3;
                    }
                }
                uint32_t r1 = 2 * u, r2 = 2 * u + 1;
                emit_read(&r, o, frag, need, seq + off[r1], (uint32_t)(off[r1 + 1] - off[r1]));
                /* read 2: reverse complement of the fragment's far end (template runs from fragment
                 * position F-1 leftwards) */
                uint8_t *t2 = frag + need;
                for (uint64_t q = 0; q < F; ++q) t2[q] = comp(frag[F - 1 - q]);
                emit_read(&r, o, t2, F, seq + off[r2], (uint32_t)(off[r2 + 1] - off[r2]));
                if (origin) {
                    origin[r1] = start | ((uint64_t)strand << 63);
                    origin[r2] = start | ((uint64_t)(!strand) << 63);
                }
            } else {
                uint32_t L = (uint32_t)(off[u + 1] - off[u]);
                uint64_t need = (uint64_t)L + 16;
                if (need > ref_len) need = ref_len;
                if (need > cap) { free(frag); cap = need; frag = (uint8_t *)malloc(cap); }
                uint64_t start = rng_below(&r, ref_len - need + 1);
                int strand = (int)(rng_u64(&r) >> 63);
                for (uint64_t q = 0; q < need; ++q)
                    frag[q] = strand ? comp(ref[start + need - 1 - q]) : ref[start + q];
                emit_read(&r, o, frag, need, seq + off[u], L);
                if (origin) origin[u] = start | ((uint64_t)strand << 63);
            }
        }
        free(frag);
    }
}
