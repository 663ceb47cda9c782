/*
 * mt4g.h — C ABI of the B300 Kolmogorov-Smirnov change-point engine.
 *
 * The engine evaluates series of latency samples the way the size benchmarks of
 * MT4G (arXiv 2511.05958) evaluate theirs: a series is a 2D array with one row per
 * array-size step and the first m measured latencies of that step in the row
 * (paper Sec. IV-B-1, step (4)); every step index is a candidate change point; the
 * two-sample Kolmogorov-Smirnov statistic D = max_x |F(x) - G(x)| (Sec. II-C-1)
 * between the samples left and right of a split decides it, and its significance
 * is reported (Sec. IV-B-1 (4)).  Binary segmentation repeats the test inside the
 * two parts to find every boundary (the segmentation criterion of Sec. II-C).
 *
 * Conventions shared by every call
 *   - samples: DEVICE pointer, uint32, all series concatenated, each step-major:
 *     sample j of step t of series s is samples[offsets[s] + t*m_s + j].
 *   - offsets: HOST int64[S+1], offsets[0] = 0, non-decreasing.
 *     steps:   HOST int32[S], T_s = steps[s] with 2 <= T_s <= MT4G_MAX_STEPS;
 *     m_s = (offsets[s+1] - offsets[s]) / T_s must be an integer >= 1 and
 *     T_s * m_s <= MT4G_MAX_SERIES_SAMPLES.
 *   - A change-point index k is the first step of the right part: the split
 *     compares steps [lo, k) with steps [k, hi).
 *   - D is returned exactly as an unreduced int64 pair: dnum / dden with
 *     dden = n_L * n_R (n_L = m (k - lo), n_R = m (hi - k)) and
 *     dnum = max_x |N c_L(x) - n_L C(x)|, N = n_L + n_R, c_L and C the counts of
 *     left and pooled samples <= x.  The split maximises D; ties go to the
 *     smallest k.
 *   - p is the asymptotic Kolmogorov p-value Q(lambda), lambda = dnum /
 *     sqrt(N * dden) in FP64, the distribution whose first term inverts to the
 *     critical value of Eq. 1; lambda^2 > 345 gives exactly 0.
 *   - Outputs are DEVICE arrays owned by the caller.  The library never frees
 *     caller memory and keeps no pointer to it after the call returns.
 *   - Calls are asynchronous on cuda_stream (a cudaStream_t; NULL = legacy
 *     default stream).  Outputs are valid after the stream is synchronised.
 *     The return value reports host-side validation and launch errors;
 *     conditions found on the device (capacity overflow, an expired bounded
 *     wait) are returned by mt4g_wait().
 *   - A context is not thread-safe: one host thread issues its calls at a time.
 *     It owns the device workspace, which grows on demand and is reused.
 *   - There is no CPU fallback: without a usable CUDA device every call fails
 *     with MT4G_ECUDA.
 */
#ifndef MT4G_H
#define MT4G_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MT4G_OK 0
#define MT4G_EINVAL (-1)    /* bad argument: offsets, T < 2, non-integral m, alpha not in (0,1) ... */
#define MT4G_ECAPACITY (-2) /* a series had more than max_cp change points (counts stay true) */
#define MT4G_ENOMEM (-3)    /* device or pinned-host allocation failed */
#define MT4G_ECUDA (-4)     /* a CUDA runtime call failed; message in mt4g_last_error */
#define MT4G_ETIMEOUT (-5)  /* a bounded device-side wait expired; outputs are incomplete */
#define MT4G_ECHECK (-6)    /* a device consistency check (MT4G_OPT_CHECKS) failed; outputs are void */

#define MT4G_MODE_FULL 0    /* every split of every segment is evaluated */
#define MT4G_MODE_LEARNED 1 /* proposal windows + exact certification; same answers as FULL */
#define MT4G_MODE_REDUCED 2 /* Eq. 2 reduction first: one FP64 value per step, then the same test */

#define MT4G_MAX_STEPS 32768

/* Scan tile value of the run sweep: one warp walks all splits of a segment in order, moving
   one step's samples to the left part at a time.  It applies to series with at most 1536
   distinct values and to segments with m H^2 < 2^31; other segments of such series are
   scanned in 32-split slices.  Where the autotuner has no entry, every call (full, reduced or
   learned) plans it for series of at most 2^17 samples and uses it when those carry at least
   half of the call's T^2 m.  In learned calls the series the sweep takes are scanned in full
   by it (see mt4g_ks_segment); the proposal probes serve the series scanned in slices. */
#define MT4G_SCAN_SWEEP 8
#define MT4G_MAX_SERIES_SAMPLES (1LL << 30)

/* Options for mt4g_set_option. */
#define MT4G_OPT_WAIT_LIMIT_NS 1 /* bound on any device-side wait in the work queue (default 5e9 ns) */
#define MT4G_OPT_STAGE_TIMING 2  /* 1: record CUDA events between the stages of every call */
#define MT4G_OPT_SCAN_KPT 3      /* scan tile: 0 = per-series choice (default), else 1, 2 or 4
                                    groups of 32 splits per warp work item, or MT4G_SCAN_SWEEP,
                                    for every series */
#define MT4G_OPT_WINDOWS 4       /* learned mode: proposal windows per series (default 3) */
#define MT4G_OPT_HALF_WIDTH 5    /* learned mode: window half width in steps (default 16) */
#define MT4G_OPT_CONF_MIN_PPM 6  /* learned mode: series whose window mass is below this (in
                                    millionths, default 900000) take the full scan */
#define MT4G_OPT_GRAPH 7         /* 1: mt4g_ks_scan / mt4g_ks_segment run as one CUDA-graph launch.
                                    The first call with given arguments (pointers, sizes, host
                                    table contents, options, weights) is captured; identical calls
                                    replay it.  Stage timing is not recorded for graph calls. */
#define MT4G_OPT_CHECKS 8        /* 1: after the per-series sort, one extra kernel checks what the
                                    scan relies on (run table from 0 to N, strictly increasing;
                                    labels < T; labels non-decreasing inside a run); a violation
                                    makes mt4g_wait return MT4G_ECHECK.  Off by default. */
#define MT4G_OPT_SWEEP_SKIP 9    /* 1: the run sweep skips splits that an exact bound excludes: a step
                                    moves m samples, so |g_(k+j) - g_k| <= j m H (g = max_x |H c_L -
                                    (k - lo) C|); a split whose bound from the last evaluated split
                                    gives a D strictly below the best D so far is not evaluated (its
                                    samples still move).  The answers are those of the full scan;
                                    mt4g_last_work counts only the evaluated pairs.  Off by default. */
#define MT4G_OPT_LEARNED_WINDOWS 10 /* 1: in MT4G_MODE_LEARNED, a series the run sweep takes and whose
                                    window mass reaches the threshold is scanned only at the splits
                                    of its windows (|k - c| <= half width), with no certification:
                                    the exact D of those splits decides each segment, a segment
                                    without window splits is not split, and a series whose top
                                    level has no significant window split falls back to the full
                                    scan (fallback = 1).  The answers can then differ from
                                    MT4G_MODE_FULL where a change point lies outside every window;
                                    the agreement is measured, not guaranteed.  Off by default. */

typedef struct mt4g_ctx mt4g_ctx;

/* Create a context on CUDA device `device`.  *ctx receives the handle.
 * Returns MT4G_OK, MT4G_ECUDA (no such device / no driver) or MT4G_ENOMEM. */
int mt4g_create(mt4g_ctx **ctx, int device);

/* Release the context and its device workspace.  Waits for its work to finish. */
void mt4g_destroy(mt4g_ctx *ctx);

/* Message for the most recent failing call on this context ("" if none).
 * The string is owned by the context and valid until its next call. */
const char *mt4g_last_error(const mt4g_ctx *ctx);

/* Synchronise the stream of the most recent call and return its device-side
 * status: MT4G_OK, MT4G_ECAPACITY (some cp_count > max_cp) or MT4G_ETIMEOUT. */
int mt4g_wait(mt4g_ctx *ctx);

/* Set a context option (see MT4G_OPT_*).  Returns MT4G_OK or MT4G_EINVAL. */
int mt4g_set_option(mt4g_ctx *ctx, int option, int64_t value);

/*
 * One top-level test per series over every split k in [1, T_s - 1]
 * (paper Sec. IV-B-1 (4): every index of the series is a potential change point;
 * Sec. II-C-1: D = max_x |F(x) - G(x)|).
 * Outputs (DEVICE, [S]): k_out = best split, dnum_out / dden_out = its exact D,
 * p_out = its p-value.
 * mode: MT4G_MODE_FULL on the raw samples, or MT4G_MODE_REDUCED on the Eq. 2
 * values S_t = sqrt(sum_j (r_tj - min r)^2) (one sample per step, m = 1 in the
 * D and p formulas).
 */
int mt4g_ks_scan(mt4g_ctx *ctx, const uint32_t *samples, const int64_t *offsets, const int32_t *steps,
                 int64_t S, int32_t mode, int32_t *k_out, int64_t *dnum_out, int64_t *dden_out,
                 double *p_out, void *cuda_stream);

/*
 * Binary segmentation of every series (segmentation criterion of Sec. II-C,
 * applied split by split with the test of Sec. IV-B-1 (4)): scan [lo, hi); if
 * p <= alpha accept the best split k and recurse into [lo, k) and [k, hi).  Each
 * side of a split keeps at least min_seg >= 1 steps; shorter segments are not
 * split.  No multiple-testing correction.
 * Outputs (DEVICE): cp_count[S] = number of change points found in series s
 * (the true count even above max_cp); cp_idx, dnum, dden, p [S * max_cp]: the
 * first min(count, max_cp) change points of series s in ascending order, each
 * with the D and p of the split that created it; unused slots are -1, 0, 0, 1.0.
 * If some count exceeds max_cp, mt4g_wait() returns MT4G_ECAPACITY.
 * mode: MT4G_MODE_FULL or MT4G_MODE_REDUCED (as in mt4g_ks_scan), or MT4G_MODE_LEARNED:
 *   the proposal network (weights from mt4g_cnn_load / mt4g_cnn_init; m <= 256) gives
 *   each series windows and a confidence (mt4g_propose).  Series below the confidence
 *   threshold take the full scan, and so do series the run sweep takes (MT4G_SCAN_SWEEP):
 *   its cost per split is below that of the probes; when it takes every series of the call,
 *   the proposal kernels return at once (no windows are computed).  For the others every
 *   segment is first scanned exactly
 *   at the windows' splits and at up to 32 grid splits; each gap between grid splits gets
 *   a bound on D from its two end columns, and the gaps whose bound might reach the best
 *   D found are scanned exactly.  The results are therefore those of MT4G_MODE_FULL.
 *   With MT4G_OPT_LEARNED_WINDOWS the series the run sweep takes are instead scanned only
 *   at their window splits (see the option), and the answers are those of the windows.
 * fallback: DEVICE int32 [S] or NULL; 1 where the series took the full scan (low
 *   confidence, the run sweep without MT4G_OPT_LEARNED_WINDOWS, or a window-only top level
 *   without a significant split; always 0 outside learned mode).
 * crit: DEVICE double [S * max_cp] or NULL; beside each reported change point, the critical
 *   value of D at level alpha for the two sample sizes of the split that created it (Eq. 1,
 *   read with the minus sign its printed radicand lost and the natural log):
 *     crit = sqrt(-1/2 ln(alpha / 2) (n_L + n_R) / (n_L n_R)),
 *   n_L = m (k - lo), n_R = m (hi - k) (m = 1 in MT4G_MODE_REDUCED), evaluated in FP64 in that
 *   order with ln(alpha / 2) taken once on the host; the paper reports this threshold as the
 *   confidence of a boundary (Sec. IV-B-1 (4)).  Unused slots are 0.
 */
int mt4g_ks_segment(mt4g_ctx *ctx, const uint32_t *samples, const int64_t *offsets, const int32_t *steps,
                    int64_t S, double alpha, int32_t min_seg, int32_t max_cp, int32_t mode,
                    int32_t *cp_count, int32_t *cp_idx, int64_t *dnum, int64_t *dden, double *p,
                    int32_t *fallback, double *crit, void *cuda_stream);

/*
 * mt4g_ks_segment with the samples in HOST memory (the same segmentation and results).
 * The batch is cut into chunks of consecutive series of at most chunk_samples samples each
 * (<= 0: an eighth of the batch, at least 2^24; a longer series is a chunk by itself).  Chunk c + 1 is copied to the device on
 * the context's copy stream while chunk c is segmented on cuda_stream, through two device
 * staging buffers the context keeps, so the host-to-device transfer overlaps the computation;
 * give samples_host in page-locked memory (cudaMallocHost / cudaHostRegister) for the copies
 * to run asynchronously.  offsets/steps are HOST tables as for mt4g_ks_segment; the outputs
 * are DEVICE arrays indexed by the global series number.  Asynchronous like every call:
 * samples_host must stay valid and unchanged until mt4g_wait() returns, and mt4g_wait()
 * reports the combined device-side status of all chunks.  CUDA-graph replay does not apply.
 * No counterpart in the paper (it is the input path of a batched service).
 */
int mt4g_ks_segment_host(mt4g_ctx *ctx, const uint32_t *samples_host, const int64_t *offsets, const int32_t *steps,
                         int64_t S, double alpha, int32_t min_seg, int32_t max_cp, int32_t mode,
                         int64_t chunk_samples, int32_t *cp_count, int32_t *cp_idx, int64_t *dnum, int64_t *dden,
                         double *p, int32_t *fallback, double *crit, void *cuda_stream);

/* ------------------------------------------------------------------ learned proposal
 *
 * The paper scans every index (Sec. IV-B-1 (4)) and notes that candidate change points
 * can be shortlisted first to save computation, a step MT4G omits because its datasets
 * are small (Sec. IV-B-1, after step (4)).  The calls below build such a shortlist with a
 * small 1D CNN over per-step summaries; the exact scan still decides every answer.
 *
 * Features (mt4g_summaries): for each step t of a series, 17 values
 *   i < 16: log2(q_i) - log2(med), q_i = the step's sorted sample at rank
 *           min(m - 1, floor((i + 0.5) m / 16)), med = the series' sorted sample at N / 2;
 *   16:     log2(1024 + 32 t) - 10 (the array size of the step);
 * values below 1 read as 1; stored as BF16 bit patterns (round to nearest even) in rows
 * of MT4G_FEAT_CHANNELS (channel 17 is zero).  Series s owns the rows
 * [R_s, R_s + T_s + 4), R_s = sum_{s' < s} (T_s' + 4); step t is row R_s + 2 + t and the two
 * rows on each side are zero.  m <= 256.
 *
 * Network: width-5 convolutions along the steps (zero padding 2), 18 -> 32 -> 32 -> 32 -> 1
 * channels, ReLU after the first three, one logit per step (13,217 trained parameters).
 * Weights are a flat FP32 vector of MT4G_CNN_PARAMS values: W1 [5][18][32], b1 [32],
 * W2 [5][32][32], b2, W3 [5][32][32], b3, W4 [5][32][1], b4 [1] (tap-major, output
 * channel fastest).  Kernels read BF16 roundings of the weights and of the activations
 * and accumulate in FP32.
 * Loss: softmax over a series' T steps, cross-entropy against the distribution uniform
 * over its change points; series with none are left out; mean over the others.
 * Training (mt4g_cnn_train_step): one batch of B series with a common T, Adam
 * (lr, beta 0.9 / 0.999, eps 1e-8, bias correction) on the FP32 master weights.
 */
#define MT4G_FEAT_CHANNELS 18
#define MT4G_CNN_PARAMS 13377

/* Per-step features of every series (layout above) into feat_out (DEVICE, BF16 bits,
 * [sum_s (T_s + 4)][18]).  Samples and host tables as for mt4g_ks_scan. */
int mt4g_summaries(mt4g_ctx *ctx, const uint32_t *samples, const int64_t *offsets, const int32_t *steps,
                   int64_t S, uint16_t *feat_out, void *cuda_stream);

/* Initialise the weights (He-uniform from splitmix64(seed), zero biases) and the Adam state. */
int mt4g_cnn_init(mt4g_ctx *ctx, uint64_t seed);
/* Copy the FP32 master weights to / from a HOST array of MT4G_CNN_PARAMS floats. */
int mt4g_cnn_get_params(mt4g_ctx *ctx, float *host_out);
int mt4g_cnn_set_params(mt4g_ctx *ctx, const float *host_in);
/* Weights file: header (magic, sizes, Adam step, CRC-32) + weights + Adam moments.
 * Loading checks the header and the checksum (MT4G_EINVAL on mismatch). */
int mt4g_cnn_save(mt4g_ctx *ctx, const char *path);
int mt4g_cnn_load(mt4g_ctx *ctx, const char *path);

/* Logits of every step: feat (DEVICE, layout above), steps (HOST int32 [S]);
 * logits_out (DEVICE float, one per feature row; pad rows are not written). */
int mt4g_cnn_forward(mt4g_ctx *ctx, const uint16_t *feat, const int32_t *steps, int64_t S, float *logits_out,
                     void *cuda_stream);

/* Loss and gradients of a batch of B series with T steps each (feat: B (T + 4) rows).
 * cp_count (DEVICE int32 [B]) and cp_idx (DEVICE int32 [B * max_cp]) give each series'
 * change points.  grad_out: DEVICE float [MT4G_CNN_PARAMS]; loss_out: DEVICE float or NULL. */
int mt4g_cnn_grads(mt4g_ctx *ctx, const uint16_t *feat, int32_t T, int64_t B, const int32_t *cp_count,
                   const int32_t *cp_idx, int32_t max_cp, float *grad_out, float *loss_out, void *cuda_stream);
/* The same forward and backward pass followed by one Adam update. */
int mt4g_cnn_train_step(mt4g_ctx *ctx, const uint16_t *feat, int32_t T, int64_t B, const int32_t *cp_count,
                        const int32_t *cp_idx, int32_t max_cp, float lr, float *loss_out, void *cuda_stream);

/* Change-point windows of every series: features, logits, softmax over the steps, then
 * n_win (<= 8) times the largest remaining logit (smallest step on ties) as a centre c,
 * removing the steps within +-half_width of it.  win_center: DEVICE int32 [S * n_win]
 * (-1 when fewer windows exist); conf: DEVICE float [S], the softmax mass of the union of
 * the windows [c - half_width, c + half_width]. */
int mt4g_propose(mt4g_ctx *ctx, const uint32_t *samples, const int64_t *offsets, const int32_t *steps, int64_t S,
                 int32_t n_win, int32_t half_width, int32_t *win_center, float *conf, void *cuda_stream);

/*
 * Scan-tile autotuner (no counterpart in the paper).  The work queue scans each segment
 * either by the run sweep (MT4G_SCAN_SWEEP, one item per segment) or in warp items of 32, 64
 * or 128 splits (the tile).  mt4g_autotune times mt4g_ks_scan with each choice on up to 256
 * series of every (floor log2 T, floor log2 m) bucket present in the batch (copied into a
 * temporary buffer) and keeps the fastest per bucket in the context; the run sweep is a
 * candidate only where it takes at least half of the bucket's series (the others would run as
 * slices inside the sweep kernel, which holds fewer warps).  Later calls use the table for
 * series of that bucket (default: the run sweep).  Synchronises the stream.  The table can be
 * written to and read from a text file; mt4g_autotune_get returns the choice (1, 2 or 4
 * groups of 32, or MT4G_SCAN_SWEEP) used for a shape.
 */
int mt4g_autotune(mt4g_ctx *ctx, const uint32_t *samples, const int64_t *offsets, const int32_t *steps, int64_t S,
                  void *cuda_stream);
int mt4g_autotune_save(mt4g_ctx *ctx, const char *path);
int mt4g_autotune_load(mt4g_ctx *ctx, const char *path);
int mt4g_autotune_get(mt4g_ctx *ctx, int32_t T, int32_t m);

/* Critical value of D at level alpha for samples of n_left and n_right values (Eq. 1, with
 * the minus sign its printed radicand lost and the natural log):
 *   d_alpha = sqrt(-1/2 ln(alpha / 2) (n_left + n_right) / (n_left n_right)),
 * the inversion of the first term 2 exp(-2 lambda^2) = alpha of the Kolmogorov series.
 * Returns -1 for alpha outside (0, 1) or a sample size below 1.  Host function. */
double mt4g_critical_value(double alpha, int64_t n_left, int64_t n_right);

/* Load-latency statistics of every series (paper Sec. IV-C: MT4G reports the average as the
 * main result, with p50, p95 and the standard deviation), over all T_s * m_s samples of a
 * series; samples and host tables as for mt4g_ks_scan.  Definitions (the paper names the
 * statistics, not their estimators):
 *   mean_out[s] = (sum x) / N, the exact integer sum rounded once to FP64;
 *   p50_out[s], p95_out[s] = sorted[ceil(q N) - 1] for q = 1/2 and 95/100 (nearest rank);
 *   std_out[s] = sqrt((N sum x^2 - (sum x)^2) / N^2), the population standard deviation with
 *   an exact 128-bit numerator rounded once to FP64 (nearest, ties to even).
 * Outputs: DEVICE double [S], uint32 [S], uint32 [S], double [S].  The order statistics come
 * from the same per-series sort the scan uses; the sums from one more read of the samples. */
int mt4g_latency_stats(mt4g_ctx *ctx, const uint32_t *samples, const int64_t *offsets, const int32_t *steps,
                       int64_t S, double *mean_out, uint32_t *p50_out, uint32_t *p95_out, double *std_out,
                       void *cuda_stream);

/*
 * Allocation-free variant of mt4g_ks_scan (no counterpart in the paper).
 *
 * For callers that cannot allocate device (or host) memory: code running inside a memory
 * pool or arena it does not own, or processes that forbid allocation after start-up.  Same
 * arguments and results as mt4g_ks_scan in MT4G_MODE_FULL (top-level test over every split
 * of every series), but without a context: all scratch comes from one static device array
 * of MT4G_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds until the process
 * exits, and host tables from a static host buffer.  Limits: S <= MT4G_NOALLOC_MAX_SERIES,
 * total samples <= MT4G_NOALLOC_MAX_SAMPLES, total steps <= MT4G_NOALLOC_MAX_STEPS; beyond
 * them the call returns MT4G_EINVAL before touching the GPU.  It runs on the current CUDA
 * device.  The array keeps the last call's contents and is shared by all calls on a device:
 * the call clears what must start at zero, but calls whose GPU work overlaps (different
 * streams or host threads) race on it.  The first call on a device looks up the array's
 * address (cudaGetSymbolAddress).  The call is synchronous: it returns after the outputs are
 * written (or, on a failed enqueue, after the work already enqueued has finished), with
 * MT4G_OK, MT4G_EINVAL, MT4G_ECUDA, MT4G_ETIMEOUT or MT4G_ECAPACITY.
 */
#define MT4G_NOALLOC_SCRATCH_BYTES (12u << 20)
#define MT4G_NOALLOC_MAX_SERIES 4096
#define MT4G_NOALLOC_MAX_SAMPLES (1 << 19)
#define MT4G_NOALLOC_MAX_STEPS (1 << 16)
int mt4g_ks_scan_noalloc(const uint32_t *samples, const int64_t *offsets, const int32_t *steps, int64_t S,
                         int32_t *k_out, int64_t *dnum_out, int64_t *dden_out, double *p_out, void *cuda_stream);

/*
 * Measurement helpers (no counterpart in the paper; they instrument the calls above).
 *
 * mt4g_stage_times: with MT4G_OPT_STAGE_TIMING on, each call records CUDA events on its
 * stream between its stages; this writes, for the last n calls (at most 64, oldest
 * first), 5 durations in ms per call: [table upload, reduce + sort + run table,
 * features + network + windows (learned mode, else 0), work-queue kernel, collect].  Synchronises on those events.  Returns the number of calls written
 * (>= 0) or a negative error code.
 *
 * mt4g_last_work: after mt4g_wait(), the number of (split k, distinct value) pairs the
 * last call evaluated, summed over all scanned segments (the scan's algorithmic work).
 */
int mt4g_stage_times(mt4g_ctx *ctx, double *ms_out, int32_t max_calls);
int mt4g_last_work(mt4g_ctx *ctx, int64_t *evals);
/* mt4g_int32_peak: the measured ceiling of the scan's inner step.  Runs the step's integer
 * mix (two multiply-adds, an absolute value, a max: 4 ops per (split, distinct value)
 * evaluation) with independent chains on every SM of CUDA device `device` for a few ms, and
 * writes the best of three timed launches in 10^12 integer ops/s to *tops_out (host).
 * Synchronous; uses its own stream; allocates nothing.  MT4G_OK or MT4G_ECUDA. */
int mt4g_int32_peak(int device, double *tops_out);
/* Failure-detection self-test (no counterpart in the paper): runs the work-queue kernel
 * over a queue that claims one pending item and never publishes it, with every wait bounded
 * by limit_ns (<= 2e9).  mt4g_wait() must then return MT4G_ETIMEOUT, and the context stays
 * usable for the next call. */
int mt4g_selftest_wait_timeout(mt4g_ctx *ctx, int64_t limit_ns, void *cuda_stream);
/* After mt4g_wait() on a learned call: out[0] = segments decided by their probe group,
 * out[1] = segments that needed refinement slices, out[2] = probe groups pushed. */
int mt4g_learned_stats(mt4g_ctx *ctx, int64_t *out);
/* After mt4g_wait(), for the last call: out[0] = segments scanned by the run sweep
 * (MT4G_SCAN_SWEEP); out[1] = samples whose run index the sort wrote for the sweep; out[2] = of
 * those, samples of series the sort handled by counting values instead of radix-sorting them
 * (no sorted labels needed: value span <= 11552, every segment swept); out[3] = series of a
 * sweep call that the sweep does not take (when 0, a learned call skips its proposals).  No
 * counterpart in the paper (work accounting for the rooflines). */
int mt4g_last_sweep(mt4g_ctx *ctx, int64_t *out);

#ifdef __cplusplus
}
#endif
#endif /* MT4G_H */
