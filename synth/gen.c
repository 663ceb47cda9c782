/*
 * Seeded synthetic latency-series generator.
 *
 * This module only produces inputs: series of uint32 cycle counts, T array-size
 * steps per series with m samples per step, stored step-major
 * (samples[off + t*m + j]), in the shape of the 2D result array of the size
 * benchmarks (one row per array size, the first N latencies of each kept;
 * paper Sec. IV-B-1, step (4)).  It holds none of the change-point method's
 * arithmetic and is shared by the CPU oracle, the tests and the benchmark.
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018) seeded from
 * splitmix64 (Steele, Lea & Flood, 2014).  Every (seed, series, stream) triple
 * has its own stream: stream 0xFFFFFFFF draws the series parameters (T, m,
 * change points, level medians), stream t draws the m samples of step t.  The
 * output is therefore identical for any thread count or series chunking.
 *
 * Distributions: Poisson by Knuth's product-of-uniforms method, normal by
 * Box-Muller (cosine branch), lognormal exp(mu + sigma z), Pareto
 * x_m * U^(-1/a).  Continuous draws are rounded with llround and clamped to
 * [1, 2^32 - 1].
 *
 * Workloads (cfg):
 *   1  one series, T=64, m=32: steps 0-39 are 32+Poisson(2), steps 40-63 are
 *      210+Poisson(6); each sample is replaced w.p. 0.01 by U{1000..5000}.
 *   2  T=512, m=128, three change points cp_i = 16 i + u_(i) with u sorted
 *      uniform integers in [0, 448] (every segment >= 16 steps); level
 *      medians 35, 300, 800, 1100 with lognormal sigma .05, .05, .08, .10;
 *      each sample replaced w.p. 0.005 by U{2000..10000}.
 *   3  T ~ U{32..4096}, m ~ U{8,16,64,256}, #cp ~ U{0..4} clipped to
 *      floor(T/16)-1, placed as in workload 2 with minimum segment 16; base median
 *      35, each next median multiplied by r, r log-uniform in [1.01, 30];
 *      sigma .05; each sample replaced w.p. 0.01 by a Pareto(1.5) draw with
 *      x_m = the level median.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SYN_MAX_CP 8

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t sm64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_next(rng_t *r) {
    uint64_t *s = r->s;
    uint64_t out = rotl64(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return out;
}

static void rng_seed(rng_t *r, uint64_t seed, uint64_t series, uint64_t stream) {
    uint64_t x = seed * 0x9E3779B97F4A7C15ULL ^ (series + 1) * 0xD1B54A32D192ED03ULL ^
                 (stream + 1) * 0x8CB92BA72F3D8DD7ULL;
    for (int i = 0; i < 4; i++) r->s[i] = sm64_next(&x);
}

/* uniform double in (0, 1] */
static double u01(rng_t *r) { return ((rng_next(r) >> 11) + 1) * 0x1.0p-53; }

/* uniform integer in [a, b] */
static int64_t uint_in(rng_t *r, int64_t a, int64_t b) {
    double u = (rng_next(r) >> 11) * 0x1.0p-53; /* [0,1) */
    int64_t v = a + (int64_t)(u * (double)(b - a + 1));
    return v > b ? b : v;
}

static int poisson_knuth(rng_t *r, double lambda) {
    double L = exp(-lambda), p = 1.0;
    int k = 0;
    do {
        k++;
        p *= u01(r);
    } while (p > L);
    return k - 1;
}

static double normal_bm(rng_t *r) {
    double u1 = u01(r), u2 = u01(r);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2);
}

static uint32_t clamp_round(double v) {
    if (!(v >= 1.0)) return 1u;
    if (v >= 4294967295.0) return 4294967295u;
    long long q = llround(v);
    if (q < 1) q = 1;
    if (q > 4294967295LL) q = 4294967295LL;
    return (uint32_t)q;
}

typedef struct {
    int32_t T, m, ncp;
    int32_t cp[SYN_MAX_CP];
    double mu[SYN_MAX_CP + 1];    /* log of level median */
    double sigma[SYN_MAX_CP + 1]; /* lognormal sigma */
} sparams;

static int cmp_i64(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* cps: c sorted uniform integers u in [0, T - 16(c+1)], cp_i = 16 (i+1) + u_(i) */
static void place_cps(rng_t *r, int32_t T, int32_t c, int32_t *cp) {
    int64_t u[SYN_MAX_CP];
    int64_t span = (int64_t)T - 16 * (int64_t)(c + 1);
    for (int i = 0; i < c; i++) u[i] = uint_in(r, 0, span);
    qsort(u, c, sizeof(int64_t), cmp_i64);
    for (int i = 0; i < c; i++) cp[i] = (int32_t)(16 * (i + 1) + u[i]);
}

static int series_params(int cfg, uint64_t seed, int64_t s, sparams *P) {
    rng_t r;
    rng_seed(&r, seed, (uint64_t)s, 0xFFFFFFFFull);
    memset(P, 0, sizeof(*P));
    if (cfg == 1) {
        P->T = 64;
        P->m = 32;
        P->ncp = 1;
        P->cp[0] = 40;
    } else if (cfg == 2) {
        static const double med[4] = {35.0, 300.0, 800.0, 1100.0};
        static const double sig[4] = {0.05, 0.05, 0.08, 0.10};
        P->T = 512;
        P->m = 128;
        P->ncp = 3;
        place_cps(&r, 512, 3, P->cp);
        for (int i = 0; i < 4; i++) {
            P->mu[i] = log(med[i]);
            P->sigma[i] = sig[i];
        }
    } else if (cfg == 3) {
        static const int32_t ms[4] = {8, 16, 64, 256};
        P->T = (int32_t)uint_in(&r, 32, 4096);
        P->m = ms[uint_in(&r, 0, 3)];
        int32_t c = (int32_t)uint_in(&r, 0, 4);
        int32_t cmax = P->T / 16 - 1;
        if (c > cmax) c = cmax;
        P->ncp = c;
        place_cps(&r, P->T, c, P->cp);
        P->mu[0] = log(35.0);
        P->sigma[0] = 0.05;
        for (int i = 1; i <= c; i++) {
            double lr = log(1.01) + u01(&r) * (log(30.0) - log(1.01));
            P->mu[i] = P->mu[i - 1] + lr;
            P->sigma[i] = 0.05;
        }
    } else {
        return -1;
    }
    return 0;
}

static void fill_series(int cfg, uint64_t seed, int64_t s, const sparams *P, uint32_t *x) {
    int32_t level = 0;
    for (int32_t t = 0; t < P->T; t++) {
        while (level < P->ncp && t >= P->cp[level]) level++;
        rng_t r;
        rng_seed(&r, seed, (uint64_t)s, (uint64_t)t);
        uint32_t *row = x + (int64_t)t * P->m;
        for (int32_t j = 0; j < P->m; j++) {
            double u = u01(&r);
            uint32_t v;
            if (cfg == 1) {
                if (u <= 0.01)
                    v = (uint32_t)uint_in(&r, 1000, 5000);
                else if (level == 0)
                    v = 32u + (uint32_t)poisson_knuth(&r, 2.0);
                else
                    v = 210u + (uint32_t)poisson_knuth(&r, 6.0);
            } else if (cfg == 2) {
                if (u <= 0.005)
                    v = (uint32_t)uint_in(&r, 2000, 10000);
                else
                    v = clamp_round(exp(P->mu[level] + P->sigma[level] * normal_bm(&r)));
            } else {
                if (u <= 0.01)
                    v = clamp_round(exp(P->mu[level]) * pow(u01(&r), -1.0 / 1.5));
                else
                    v = clamp_round(exp(P->mu[level] + P->sigma[level] * normal_bm(&r)));
            }
            row[j] = v;
        }
    }
}

/* Per-series shapes and truth.  T, m: [count]; ncp: [count]; cps: [count * 8]. */
int mt4g_synth_params(int cfg, uint64_t seed, int64_t series_begin, int64_t count, int32_t *T,
                      int32_t *m, int32_t *ncp, int32_t *cps) {
    for (int64_t i = 0; i < count; i++) {
        sparams P;
        if (series_params(cfg, seed, series_begin + i, &P)) return -1;
        if (T) T[i] = P.T;
        if (m) m[i] = P.m;
        if (ncp) ncp[i] = P.ncp;
        if (cps)
            for (int c = 0; c < SYN_MAX_CP; c++) cps[i * SYN_MAX_CP + c] = c < P.ncp ? P.cp[c] : -1;
    }
    return 0;
}

typedef struct {
    int cfg;
    uint64_t seed;
    int64_t series_begin, lo, hi;
    const int64_t *offsets;
    uint32_t *samples;
    int err;
} job_t;

static void *fill_worker(void *arg) {
    job_t *J = (job_t *)arg;
    for (int64_t i = J->lo; i < J->hi; i++) {
        sparams P;
        if (series_params(J->cfg, J->seed, J->series_begin + i, &P)) {
            J->err = -1;
            return NULL;
        }
        if (J->offsets[i + 1] - J->offsets[i] != (int64_t)P.T * P.m) {
            J->err = -2;
            return NULL;
        }
        fill_series(J->cfg, J->seed, J->series_begin + i, &P, J->samples + J->offsets[i]);
    }
    return NULL;
}

/* Fill series [series_begin, series_begin+count).  offsets[0..count] are element
 * offsets into samples (offsets[i+1]-offsets[i] must equal T_i*m_i).  Series are
 * dealt to nthreads workers in contiguous blocks; the output does not depend on
 * nthreads.  Returns 0, -1 (bad cfg) or -2 (offsets do not match the shapes). */
int mt4g_synth_fill(int cfg, uint64_t seed, int64_t series_begin, int64_t count,
                    const int64_t *offsets, uint32_t *samples, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (count < nthreads) nthreads = count > 0 ? (int)count : 1;
    pthread_t th[256];
    job_t jobs[256];
    for (int w = 0; w < nthreads; w++) {
        jobs[w].cfg = cfg;
        jobs[w].seed = seed;
        jobs[w].series_begin = series_begin;
        jobs[w].lo = count * w / nthreads;
        jobs[w].hi = count * (w + 1) / nthreads;
        jobs[w].offsets = offsets;
        jobs[w].samples = samples;
        jobs[w].err = 0;
    }
    for (int w = 1; w < nthreads; w++) pthread_create(&th[w], NULL, fill_worker, &jobs[w]);
    fill_worker(&jobs[0]);
    for (int w = 1; w < nthreads; w++) pthread_join(th[w], NULL);
    for (int w = 0; w < nthreads; w++)
        if (jobs[w].err) return jobs[w].err;
    return 0;
}
