/*
 * CPU oracle for Kolmogorov-Smirnov change-point detection over latency series.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header or table with
 * the CUDA path, and it is deliberately plain and slow: single pass per split,
 * straight from the definitions below, so that a reader can check it against the
 * paper by eye.
 *
 * What it computes (paper Sec. II-C-1 and Sec. IV-B-1, step (4)):
 *   A series holds T array-size steps with m latency samples each, stored
 *   step-major (x[t*m + j]).  For a segment [lo, hi) of steps and a split k with
 *   lo < k < hi, the left sample L pools steps [lo, k) and the right sample R
 *   pools steps [k, hi) (the change-point index is the first step of the right
 *   part).  With n_L = m (k - lo), n_R = m (hi - k), N = n_L + n_R, the two-sample
 *   statistic is D = max_x |F_L(x) - F_R(x)| (Sec. II-C-1), where F are the
 *   empirical CDFs.  Writing c_L(x) = #{v in L : v <= x} and
 *   C(x) = #{v in L u R : v <= x}, one has c_R = C - c_L and therefore
 *       D = max_x |N c_L(x) - n_L C(x)| / (n_L n_R) = num / den,
 *   held exactly as int64 (num, den = n_L n_R), unreduced.  x ranges over the
 *   distinct pooled values; the ECDFs are read only after all samples equal to x
 *   are counted (ties).
 *   Every index of the series is a candidate change point (Sec. IV-B-1 (4)); the
 *   chosen split maximises D over k, ties going to the smallest k; D values are
 *   compared as num_a den_b vs num_b den_a in 128-bit integers.
 *
 * p-value: the asymptotic Kolmogorov distribution that also gives Eq. 1's
 *   critical value.  lambda = num / sqrt(N * den) (= sqrt(n_L n_R / N) D), no
 *   small-sample correction (Eq. 1 has none), and
 *     Q(lambda) = 2 sum_{j>=1} (-1)^(j-1) exp(-2 j^2 lambda^2)        lambda >= 1.18
 *     Q(lambda) = 1 - sqrt(2 pi)/lambda sum_{j>=1} exp(-(2j-1)^2 pi^2 / (8 lambda^2))
 *                                                                     lambda <  1.18
 *   (the two standard forms of the Kolmogorov survival function; the switch at
 *   1.18 is the usual Numerical Recipes choice).  Terms are summed until a term
 *   falls below 1e-17 of the running sum, or for 100 terms.  lambda = 0 gives 1;
 *   lambda^2 > 345 gives 0 (the first term 2 exp(-690) is below 1e-299), so no
 *   subnormal is ever produced; the result is clamped to [0, 1].
 *
 * Critical value (Eq. 1, whose printed radicand has a lost minus sign): read as
 *   d_alpha = sqrt(-1/2 ln(alpha/2) (n + m) / (n m)), the inversion of the first
 *   series term 2 exp(-2 lambda^2) = alpha.
 *
 * Binary segmentation (the segmentation criterion V(tau, S) of Sec. II-C, found
 *   split by split): scan [lo, hi); if p <= alpha accept k and recurse on [lo, k)
 *   and [k, hi); a segment shorter than 2 min_seg steps is not split and each side
 *   of a split keeps at least min_seg steps.  No multiple-testing correction.
 *   Change points are reported in ascending order, each with the (num, den, p)
 *   of the split that created it; if there are more than max_cp, the first max_cp
 *   are written and the true count is returned.
 *
 * Geometric-mapping reduction (Eq. 2): S_t = sqrt(sum_j (r_tj - min r)^2), with
 *   min r the global minimum of the series; in the reduced variant each step is one
 *   scalar sample (m = 1) and the same scan runs over the T reduced values.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ECAPACITY (-2)
#define ORC_ENOMEM (-3)

typedef struct {
    uint32_t v; /* latency value */
    int32_t t;  /* step label */
} sample_t;

static int cmp_sample(const void *a, const void *b) {
    const sample_t *x = (const sample_t *)a, *y = (const sample_t *)b;
    if (x->v != y->v) return x->v < y->v ? -1 : 1;
    return (x->t > y->t) - (x->t < y->t); /* equal values keep step order */
}

/* Sort the T*m samples of one series by value; equal values in step order.
 * Outputs the sorted values and their step labels. */
int oracle_sort_series(const uint32_t *x, int32_t T, int32_t m, uint32_t *sv, int32_t *st) {
    int64_t N = (int64_t)T * m;
    sample_t *a = (sample_t *)malloc((size_t)(N > 0 ? N : 1) * sizeof(sample_t));
    if (!a) return ORC_ENOMEM;
    for (int64_t i = 0; i < N; i++) {
        a[i].v = x[i];
        a[i].t = (int32_t)(i / m);
    }
    qsort(a, (size_t)N, sizeof(sample_t), cmp_sample);
    for (int64_t i = 0; i < N; i++) {
        sv[i] = a[i].v;
        st[i] = a[i].t;
    }
    free(a);
    return ORC_OK;
}

/* D_a > D_b, i.e. num_a / den_a > num_b / den_b, compared exactly. */
static int d_greater(int64_t num_a, int64_t den_a, int64_t num_b, int64_t den_b) {
    unsigned __int128 l = (unsigned __int128)(uint64_t)num_a * (uint64_t)den_b;
    unsigned __int128 r = (unsigned __int128)(uint64_t)num_b * (uint64_t)den_a;
    return l > r;
}

/*
 * All-splits scan of segment [lo, hi) of one series, from its sorted samples
 * (keys: the sample values, or the Eq. 2 reduced values' bit patterns).
 * Splits k in [lo + min_seg, hi - min_seg].  For every k, one pass over the
 * segment's sorted samples accumulates c_L and C and takes |N c_L - n_L C| at
 * the end of each run of equal values.  Writes the best k (smallest on ties)
 * and its exact (num, den).  Returns ORC_EINVAL if there is no admissible split.
 */
static int scan_keys(const uint64_t *key, const int32_t *st, int64_t N_series, int32_t m, int32_t lo,
                     int32_t hi, int32_t min_seg, int32_t *k_out, int64_t *num_out, int64_t *den_out) {
    if (min_seg < 1 || m < 1 || hi - lo < 2 * min_seg) return ORC_EINVAL;
    /* the segment's samples, still in value order */
    int64_t n = 0;
    for (int64_t i = 0; i < N_series; i++)
        if (st[i] >= lo && st[i] < hi) n++;
    uint64_t *v = (uint64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(uint64_t));
    int32_t *t = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!v || !t) {
        free(v);
        free(t);
        return ORC_ENOMEM;
    }
    n = 0;
    for (int64_t i = 0; i < N_series; i++)
        if (st[i] >= lo && st[i] < hi) {
            v[n] = key[i];
            t[n] = st[i];
            n++;
        }

    int32_t best_k = -1;
    int64_t best_num = 0, best_den = 1;
    for (int32_t k = lo + min_seg; k <= hi - min_seg; k++) {
        int64_t nL = (int64_t)m * (k - lo), nR = (int64_t)m * (hi - k), NN = nL + nR;
        int64_t cL = 0, C = 0, num = 0;
        for (int64_t i = 0; i < n; i++) {
            C += 1;
            if (t[i] < k) cL += 1;
            if (i == n - 1 || v[i + 1] != v[i]) { /* end of a run of equal values */
                int64_t f = NN * cL - nL * C;
                if (f < 0) f = -f;
                if (f > num) num = f;
            }
        }
        int64_t den = nL * nR;
        if (best_k < 0 || d_greater(num, den, best_num, best_den)) {
            best_k = k;
            best_num = num;
            best_den = den;
        }
    }
    free(v);
    free(t);
    *k_out = best_k;
    *num_out = best_num;
    *den_out = best_den;
    return ORC_OK;
}

int oracle_scan_segment(const uint32_t *sv, const int32_t *st, int64_t N_series, int32_t m, int32_t lo,
                        int32_t hi, int32_t min_seg, int32_t *k_out, int64_t *num_out, int64_t *den_out) {
    uint64_t *key = (uint64_t *)malloc((size_t)(N_series > 0 ? N_series : 1) * sizeof(uint64_t));
    if (!key) return ORC_ENOMEM;
    for (int64_t i = 0; i < N_series; i++) key[i] = sv[i];
    int rc = scan_keys(key, st, N_series, m, lo, hi, min_seg, k_out, num_out, den_out);
    free(key);
    return rc;
}

/* Kolmogorov survival function Q(lambda) = P(K > lambda). */
double oracle_kolmogorov_q(double lam) {
    const double PI2 = 9.8696044010893586188; /* pi^2 */
    const double SQRT_2PI = 2.5066282746310005024;
    if (!(lam > 0.0)) return 1.0;
    double l2 = lam * lam;
    if (l2 > 345.0) return 0.0;
    double q;
    if (lam < 1.18) {
        double s = 0.0;
        for (int j = 1; j <= 100; j++) {
            double o = (double)(2 * j - 1);
            double term = exp(-(o * o) * PI2 / (8.0 * l2));
            s += term;
            if (term < 1e-17 * s) break;
        }
        q = 1.0 - SQRT_2PI / lam * s;
    } else {
        double s = 0.0;
        for (int j = 1; j <= 100; j++) {
            double jj = (double)j;
            double term = exp(-2.0 * jj * jj * l2);
            s += (j & 1) ? term : -term;
            if (term < 1e-17 * fabs(s)) break;
        }
        q = 2.0 * s;
    }
    if (q < 0.0) q = 0.0;
    if (q > 1.0) q = 1.0;
    return q;
}

/* lambda = num / sqrt(N * den): the asymptotic scaling sqrt(n_L n_R / N) D. */
double oracle_lambda(int64_t num, int64_t den, int64_t N) {
    if (num <= 0) return 0.0;
    return (double)num / sqrt((double)N * (double)den);
}

double oracle_pvalue(int64_t num, int64_t den, int64_t N) {
    return oracle_kolmogorov_q(oracle_lambda(num, den, N));
}

/* Eq. 1 critical value of D for sample sizes n and m at level alpha. */
double oracle_critical_value(double alpha, int64_t n, int64_t m) {
    return sqrt(-0.5 * log(alpha / 2.0) * (double)(n + m) / ((double)n * (double)m));
}

/* ---------------------------------------------------------------- batches */

static int check_series(const int64_t *offsets, const int32_t *steps, int64_t s, int32_t *m_out) {
    int64_t n = offsets[s + 1] - offsets[s];
    int32_t T = steps[s];
    if (T < 2 || n <= 0 || n % T != 0) return ORC_EINVAL;
    if (T > 32768) return ORC_EINVAL;
    *m_out = (int32_t)(n / T);
    return ORC_OK;
}

typedef struct {
    const uint32_t *samples;
    const int64_t *offsets;
    const int32_t *steps;
    int64_t lo, hi; /* series range of this worker */
    /* scan outputs */
    int32_t *k;
    int64_t *num, *den;
    double *p;
    /* segmentation */
    double alpha;
    int32_t min_seg, max_cp;
    int32_t *cp_count, *cp_idx;
    int64_t *cp_num, *cp_den;
    double *cp_p;
    int reduced;
    int rc;
} batch_job;

/* Eq. 2: one reduced value per step, S_t = sqrt(sum_j (r_tj - min r)^2). */
static void reduce_series(const uint32_t *x, int32_t T, int32_t m, double *S) {
    uint32_t mn = 0xFFFFFFFFu;
    for (int64_t i = 0; i < (int64_t)T * m; i++)
        if (x[i] < mn) mn = x[i];
    for (int32_t t = 0; t < T; t++) {
        double acc = 0.0;
        for (int32_t j = 0; j < m; j++) {
            double d = (double)(x[(int64_t)t * m + j] - mn);
            acc += d * d;
        }
        S[t] = sqrt(acc);
    }
}

int oracle_reduce_series(const uint32_t *x, int32_t T, int32_t m, double *S) {
    if (T < 1 || m < 1) return ORC_EINVAL;
    reduce_series(x, T, m, S);
    return ORC_OK;
}

/* Sorted (key, label) view of one series: the raw samples (key = value) or, in
 * the reduced variant, the T values of Eq. 2 (key = IEEE bit pattern, which
 * orders like the value for non-negative doubles) with m = 1. */
typedef struct {
    int64_t n;
    int32_t m;
    uint64_t *key;
    int32_t *st;
} sorted_t;

static int sort_pair64(const void *a, const void *b) {
    const uint64_t *x = (const uint64_t *)a, *y = (const uint64_t *)b;
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
    return (x[1] > y[1]) - (x[1] < y[1]);
}

static int make_sorted(const batch_job *J, int64_t s, sorted_t *out) {
    int32_t m;
    memset(out, 0, sizeof(*out));
    if (check_series(J->offsets, J->steps, s, &m)) return ORC_EINVAL;
    int32_t T = J->steps[s];
    const uint32_t *x = J->samples + J->offsets[s];
    if (!J->reduced) {
        out->n = (int64_t)T * m;
        out->m = m;
        uint32_t *sv = (uint32_t *)malloc((size_t)out->n * sizeof(uint32_t));
        out->key = (uint64_t *)malloc((size_t)out->n * sizeof(uint64_t));
        out->st = (int32_t *)malloc((size_t)out->n * sizeof(int32_t));
        if (!sv || !out->key || !out->st) {
            free(sv);
            return ORC_ENOMEM;
        }
        int rc = oracle_sort_series(x, T, m, sv, out->st);
        for (int64_t i = 0; i < out->n; i++) out->key[i] = sv[i];
        free(sv);
        return rc;
    }
    double *S = (double *)malloc((size_t)T * sizeof(double));
    uint64_t *pairs = (uint64_t *)malloc((size_t)T * 2 * sizeof(uint64_t));
    out->key = (uint64_t *)malloc((size_t)T * sizeof(uint64_t));
    out->st = (int32_t *)malloc((size_t)T * sizeof(int32_t));
    if (!S || !pairs || !out->key || !out->st) {
        free(S);
        free(pairs);
        return ORC_ENOMEM;
    }
    reduce_series(x, T, m, S);
    for (int32_t t = 0; t < T; t++) {
        uint64_t bits;
        memcpy(&bits, &S[t], sizeof(bits));
        pairs[2 * t] = bits;
        pairs[2 * t + 1] = (uint64_t)t;
    }
    qsort(pairs, (size_t)T, 2 * sizeof(uint64_t), sort_pair64);
    out->n = T;
    out->m = 1;
    for (int32_t t = 0; t < T; t++) {
        out->key[t] = pairs[2 * t];
        out->st[t] = (int32_t)pairs[2 * t + 1];
    }
    free(S);
    free(pairs);
    return ORC_OK;
}

static void free_sorted(sorted_t *x) {
    free(x->key);
    free(x->st);
}

static int scan_any(const sorted_t *X, int32_t lo, int32_t hi, int32_t min_seg, int32_t *k, int64_t *num,
                    int64_t *den) {
    return scan_keys(X->key, X->st, X->n, X->m, lo, hi, min_seg, k, num, den);
}

static void *scan_worker(void *arg) {
    batch_job *J = (batch_job *)arg;
    for (int64_t s = J->lo; s < J->hi; s++) {
        sorted_t X;
        int rc = make_sorted(J, s, &X);
        if (rc) {
            free_sorted(&X);
            J->rc = rc;
            return NULL;
        }
        int32_t T = J->steps[s];
        rc = scan_any(&X, 0, T, 1, &J->k[s], &J->num[s], &J->den[s]);
        if (rc) J->rc = rc;
        J->p[s] = oracle_pvalue(J->num[s], J->den[s], (int64_t)X.m * T);
        free_sorted(&X);
    }
    return NULL;
}

typedef struct {
    int32_t count;
    int32_t cap;
    int32_t *idx;
    int64_t *num, *den;
    double *p;
} cp_list;

/* In-order recursion, so change points come out in ascending order. */
static int segment_rec(const sorted_t *X, int32_t lo, int32_t hi, double alpha, int32_t min_seg,
                       cp_list *out) {
    if (hi - lo < 2 * min_seg) return ORC_OK;
    int32_t k;
    int64_t num, den;
    int rc = scan_any(X, lo, hi, min_seg, &k, &num, &den);
    if (rc) return rc;
    double p = oracle_pvalue(num, den, (int64_t)X->m * (hi - lo));
    if (!(p <= alpha)) return ORC_OK;
    rc = segment_rec(X, lo, k, alpha, min_seg, out);
    if (rc) return rc;
    if (out->count < out->cap) {
        out->idx[out->count] = k;
        out->num[out->count] = num;
        out->den[out->count] = den;
        out->p[out->count] = p;
    }
    out->count++;
    return segment_rec(X, k, hi, alpha, min_seg, out);
}

static void *segment_worker(void *arg) {
    batch_job *J = (batch_job *)arg;
    for (int64_t s = J->lo; s < J->hi; s++) {
        sorted_t X;
        int rc = make_sorted(J, s, &X);
        if (rc) {
            free_sorted(&X);
            J->rc = rc;
            return NULL;
        }
        int64_t b = s * J->max_cp;
        cp_list L = {0, J->max_cp, J->cp_idx + b, J->cp_num + b, J->cp_den + b, J->cp_p + b};
        rc = segment_rec(&X, 0, J->steps[s], J->alpha, J->min_seg, &L);
        if (rc) J->rc = rc;
        J->cp_count[s] = L.count;
        for (int32_t c = L.count; c < J->max_cp; c++) {
            L.idx[c] = -1;
            L.num[c] = 0;
            L.den[c] = 0;
            L.p[c] = 1.0;
        }
        free_sorted(&X);
    }
    return NULL;
}

static int run_jobs(batch_job *proto, int64_t S, int nthreads, void *(*fn)(void *)) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (S < nthreads) nthreads = S > 0 ? (int)S : 1;
    batch_job jobs[256];
    pthread_t th[256];
    for (int w = 0; w < nthreads; w++) {
        jobs[w] = *proto;
        jobs[w].lo = S * w / nthreads;
        jobs[w].hi = S * (w + 1) / nthreads;
        jobs[w].rc = 0;
    }
    for (int w = 1; w < nthreads; w++) pthread_create(&th[w], NULL, fn, &jobs[w]);
    fn(&jobs[0]);
    for (int w = 1; w < nthreads; w++) pthread_join(th[w], NULL);
    for (int w = 0; w < nthreads; w++)
        if (jobs[w].rc) return jobs[w].rc;
    return ORC_OK;
}

static int validate(const int64_t *offsets, const int32_t *steps, int64_t S) {
    if (S < 0 || !offsets || (S > 0 && !steps) || offsets[0] != 0) return ORC_EINVAL;
    for (int64_t s = 0; s < S; s++) {
        int32_t m;
        if (offsets[s + 1] < offsets[s] || check_series(offsets, steps, s, &m)) return ORC_EINVAL;
    }
    return ORC_OK;
}

/* One top-level scan per series over all splits k in [1, T-1]; series are
 * independent and dealt to nthreads workers. reduced != 0 selects Eq. 2. */
int oracle_ks_scan(const uint32_t *samples, const int64_t *offsets, const int32_t *steps, int64_t S,
                   int32_t *k, int64_t *num, int64_t *den, double *p, int reduced, int nthreads) {
    int rc = validate(offsets, steps, S);
    if (rc) return rc;
    batch_job J;
    memset(&J, 0, sizeof(J));
    J.samples = samples;
    J.offsets = offsets;
    J.steps = steps;
    J.k = k;
    J.num = num;
    J.den = den;
    J.p = p;
    J.reduced = reduced;
    return run_jobs(&J, S, nthreads, scan_worker);
}

/* Binary segmentation of every series.  Outputs: cp_count[S];
 * cp_idx, cp_num, cp_den, cp_p [S * max_cp] (unused slots: -1, 0, 0, 1.0).
 * Returns ORC_ECAPACITY if any series had more than max_cp change points. */
int oracle_ks_segment(const uint32_t *samples, const int64_t *offsets, const int32_t *steps, int64_t S,
                      double alpha, int32_t min_seg, int32_t max_cp, int32_t *cp_count, int32_t *cp_idx,
                      int64_t *cp_num, int64_t *cp_den, double *cp_p, int reduced, int nthreads) {
    int rc = validate(offsets, steps, S);
    if (rc) return rc;
    if (!(alpha > 0.0 && alpha < 1.0) || min_seg < 1 || max_cp < 0) return ORC_EINVAL;
    batch_job J;
    memset(&J, 0, sizeof(J));
    J.samples = samples;
    J.offsets = offsets;
    J.steps = steps;
    J.alpha = alpha;
    J.min_seg = min_seg;
    J.max_cp = max_cp;
    J.cp_count = cp_count;
    J.cp_idx = cp_idx;
    J.cp_num = cp_num;
    J.cp_den = cp_den;
    J.cp_p = cp_p;
    J.reduced = reduced;
    rc = run_jobs(&J, S, nthreads, segment_worker);
    if (rc) return rc;
    for (int64_t s = 0; s < S; s++)
        if (cp_count[s] > max_cp) return ORC_ECAPACITY;
    return ORC_OK;
}
