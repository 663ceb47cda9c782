// Internal declarations shared by the CUDA translation units of libmt4g.
//
// Device data layout (all in one context-owned workspace; offsets below are
// element offsets, every sub-buffer 256-byte aligned):
//   SeriesDesc desc[S]          shape of each series and its bases
//   keyA/keyB  uint32[Ntot]     radix-sort ping-pong keys (final order in keyA)
//   labA/labB  uint16[Ntot]     step labels travelling with the keys (final in labA)
//   runs       int32[Ntot + S]  per series: start of each run of equal values,
//                               runs[run_base + j], j in [0, U_s], last = N_s
//   cp_flag/num/den/p/crit [sum T]   per step: a change point accepted at that step
//   queue      WorkItem[cap] + ready[cap] + gcount[cap]   the device work queue
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mt4g.h"

namespace mt4g {

constexpr int kSortThreads = 256;  // four CTAs per SM
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;  // 2048 samples per tile

constexpr int kScanThreads = 256;  // CTA of the persistent kernel: 8 independent warps

// Run sweep of the scan: a series with at most kSweepMaxRuns distinct values gets, from the
// sort, the run index of every sample in input order (labB), and its segments are scanned
// by one warp that keeps the segment's runs in shared memory.  The kernel with the sweep
// runs CTAs of kSweepThreads (its per-warp shared memory is larger).
constexpr int kSweepMaxRuns = 1536;
constexpr int kSweepThreads = 64;

struct SeriesDesc {
    int64_t off;        // first sample of the series
    int64_t step_base;  // first per-step slot of the series (prefix sum of T)
    int64_t run_base;   // first run-table slot (off + series index)
    int32_t T;          // steps
    int32_t m;          // samples per step
    int32_t nruns;      // U_s, number of distinct values (written by the sort)
    int32_t kpt;        // scan tile: split groups of 32 per warp work item (1, 2 or 4), or 0 for
                        // the run sweep (one item per segment; slices of 32 splits when the
                        // series or segment does not qualify)
    uint32_t median;    // sorted value at index N / 2 (written by the sort)
    uint32_t p50;       // nearest-rank order statistics sorted[ceil(q N) - 1], q = 1/2 and
    uint32_t p95;       // 95/100 (written by the sort)
    int32_t flags;      // kDescNoLabels: the sort wrote run indices and the run table only
};

// SeriesDesc.flags.  A run-sweep series whose values span at most kFastSpan and whose every
// segment the sweep takes needs no sorted labels: the sort then counts values in a table
// indexed by value instead of radix-sorting, and labA is left unwritten for it.
enum : int32_t { kDescNoLabels = 1 };

// Learned-proposal feature rows: series s owns rows [row_base(s), row_base(s) + T_s + 4) of
// an [rows][kFeatC] array; step t is row row_base(s) + 2 + t and the two rows on each
// side are zero, so width-5 convolutions need no bounds checks.
constexpr int kFeatC = 18;  // 16 quantiles + step size + one zero channel
__host__ __device__ inline int64_t row_base(const SeriesDesc &d, int64_t s) { return d.step_base + 4 * s; }

// One unit of work on segment [lo, hi) of a series, member `chunk` of a group of
// `nch` items pushed together; the last member to finish combines the group.
//   kPlain:  splits [lo + min_seg + w c, ... + w - 1] with w = 32 kpt, c = chunk
//   kWindow: the 32 splits from k0 (a proposal window), exact
//   kGrid:   exact columns at up to 32 grid splits and bounds over the gaps between them
//   kRefine: the 32 splits from k0, up to klim, inside a gap that was not certified
// Splits outside [lo + min_seg, hi - min_seg] are never evaluated.
enum ItemKind : int32_t { kPlain = 0, kWindow = 1, kGrid = 2, kRefine = 3 };
struct WorkItem {
    int32_t series;
    int32_t lo;
    int32_t hi;
    int32_t chunk;
    int32_t kind_nch;  // kind | nch << 8
    int32_t k0;
    int32_t klim;
    int32_t rec;       // certification record of the segment (learned groups), else -1
};
__host__ __device__ inline int32_t item_kind(const WorkItem &w) { return w.kind_nch & 0xff; }
__host__ __device__ inline int32_t item_nch(const WorkItem &w) { return w.kind_nch >> 8; }

// Certification record of one learned segment: the grid's gaps and the best exact split.
constexpr int kMaxGrid = 32;
struct CertRecord {
    int32_t best_k;
    int32_t n_gap;
    uint64_t best_g;
    int32_t a[kMaxGrid - 1];  // gap j covers splits a[j] < k < b[j]
    int32_t b[kMaxGrid - 1];
    uint64_t ub[kMaxGrid - 1];  // bound on max_x |H c_L - (k - lo) C| for a[j] <= k <= b[j]
};

// Partial result of one group member, written over its (already consumed) queue slot.
struct ChunkResult {
    int32_t k;
    int32_t pad;
    uint64_t g;  // max_x |H c_L - (k - lo) C|; the exact numerator is m * g
};

enum : int32_t { kStatusTimeout = 1, kStatusQueueFull = 2, kStatusCapacity = 4, kStatusCheck = 8 };

struct QueueHeader {
    unsigned long long head;     // next ticket to hand out
    unsigned long long tail;     // next free slot
    long long pending;           // items pushed and not yet finished
    int32_t status;              // kStatus* bits
    int32_t pad;
    unsigned long long cap;      // slots
    unsigned long long evals;    // (k, distinct value) pairs evaluated
    unsigned long long rec_next; // certification records handed out
    unsigned long long rec_cap;
    unsigned long long refined;  // learned segments that needed refinement slices
    unsigned long long certified;  // learned segments decided by their probe group
    unsigned long long swept;      // segments scanned by the run sweep
    unsigned long long ranked;     // samples whose run index the sort wrote (sweep calls)
    unsigned long long counted;    // of those, samples of series sorted by counting (kDescNoLabels)
    unsigned long long unswept;    // series of a sweep call that the sweep does not take
};

enum RunMode : int32_t { kRunScan = 0, kRunSegment = 1, kRunLearned = 2 };

constexpr int32_t kGateNone = 0, kGateAllSwept = 1, kGateSomeUnswept = 2;

struct RunParams {
    const SeriesDesc *desc;
    const uint16_t *lab;   // sorted labels (labA)
    const uint16_t *rk;    // run index of every sample in input order (labB), or null: no sweep
    const int32_t *runs;   // run table
    QueueHeader *q;
    WorkItem *items;
    int32_t *ready;
    uint32_t *gcount;      // per group (at its first slot): members finished
    int32_t mode;          // kRunScan / kRunSegment
    int32_t min_seg;
    double alpha;
    long long wait_limit_ns;
    // scan outputs [S]
    int32_t *k_out;
    int64_t *dnum_out;
    int64_t *dden_out;
    double *p_out;
    // segmentation: per-step accepted change points
    uint8_t *cp_flag;
    int64_t *cp_num;
    int64_t *cp_den;
    double *cp_p;
    double *cp_crit;  // Eq. 1 critical value of the accepted split
    double crit_c;    // -1/2 ln(alpha / 2)
    // learned segmentation
    const int32_t *win_center;  // [S * n_win], -1 = none
    int32_t n_win;
    int32_t half;               // window slice covers [c - half, c - half + 31]
    int32_t *fallback;          // [S]: 1 = the series takes the plain path (set again by the
                                //      window-only scan when its top level is not significant)
    CertRecord *recs;
    int32_t sweep_warps;        // warps of the launch: the sweep's parts per segment follow from them
    int32_t sweep_skip;         // 1: the run sweep skips splits by the exact bound (MT4G_OPT_SWEEP_SKIP)
    int32_t win_only;           // 1: learned calls scan swept series only at their window splits
                                //    (MT4G_OPT_LEARNED_WINDOWS)
    int32_t top_parts;          // parts of a top-level run-sweep segment (planned on the host)
    int32_t gate;               // kGateNone, or which of a learned call's two queue launches works:
                                // kGateAllSwept (every series swept: the plain kernel) or
                                // kGateSomeUnswept (the learned kernel), read from q->unswept
};

// Number of slices of a segment of H steps (0 if it cannot be split).
__host__ __device__ inline int32_t seg_chunks(int32_t H, int32_t min_seg, int32_t kpt) {
    const int32_t nk = H - 2 * min_seg + 1;
    if (kpt == 0) return nk <= 0 ? 0 : 1;  // run sweep: the whole segment
    const int32_t w = 32 * kpt;
    return nk <= 0 ? 0 : (nk + w - 1) / w;
}

// Run-sweep items.  A segment the sweep takes is one item, or, when warps would otherwise be
// idle (small batches; the end of a run), up to kSweepMaxParts items that sweep consecutive
// ranges of its splits, each replaying the earlier steps' sample moves first; the group's last
// member combines their best splits.  WorkItem.rec = kSweepItem marks them, k0 .. klim is the
// part's split range.
constexpr int32_t kSweepItem = -2;
constexpr int kSweepMaxParts = 8;
constexpr int kSweepMinPartSplits = 48;

// Parts for a segment of H steps when `want` are wanted (0 if it cannot be split).
__host__ __device__ inline int32_t sweep_parts(int32_t H, int32_t min_seg, int32_t want) {
    const int32_t nk = H - 2 * min_seg + 1;
    if (nk <= 0) return 0;
    int32_t p = nk / kSweepMinPartSplits;
    p = p < 1 ? 1 : (p > kSweepMaxParts ? kSweepMaxParts : p);
    want = want < 1 ? 1 : want;
    return want < p ? want : p;
}

// Splits [k0, k1] of part c of np over the splits [A, B] of a segment.
__host__ __device__ inline void sweep_part_range(int32_t A, int32_t B, int32_t c, int32_t np, int32_t &k0,
                                                 int32_t &k1) {
    const int64_t nk = (int64_t)B - A + 1;
    k0 = A + (int32_t)(nk * c / np);
    k1 = A + (int32_t)(nk * (c + 1) / np) - 1;
}

// ---- kernels (launch wrappers live in the .cu files) ----
// sweep_stats != null (sweep calls): also write every sample's run index to labB for series
// with at most kSweepMaxRuns distinct values (the run sweep's input); sweep_stats[0] counts
// their samples, [1] those of series sorted by counting, [2] the series the sweep does not
// take (QueueHeader.ranked, .counted, .unswept).
cudaError_t launch_sort(const uint32_t *samples, SeriesDesc *desc, const int32_t *order, int64_t S,
                        uint32_t *keyA, uint32_t *keyB, uint16_t *labA, uint16_t *labB, int32_t *runs,
                        unsigned long long *sweep_stats, cudaStream_t st);

cudaError_t launch_queue_run(const RunParams &P, int grid, uint32_t epoch, cudaStream_t st);
// Top-level items: run-sweep series (kpt 0) get top_parts parts (sweep_parts), the others their
// slices; item_base[i] is the first slot of series qorder[i].
cudaError_t launch_init_items(const SeriesDesc *desc, const int32_t *qorder, const int64_t *item_base, int64_t S,
                              int32_t min_seg, int32_t top_parts, WorkItem *items, int32_t *ready, uint32_t *gcount,
                              uint32_t epoch, cudaStream_t st);
cudaError_t launch_init_learned(const RunParams &P, const float *conf, float conf_min, int32_t *fallback_out,
                                int64_t S, uint32_t epoch, cudaStream_t st);
int queue_grid(int device);        // CTAs of the slice-only kernel
int queue_grid_sweep(int device);  // CTAs of the kernel with the run sweep

// Consistency check of the sort's output (MT4G_OPT_CHECKS): run table, labels (or, for
// kDescNoLabels series, the run indices against the run lengths).  Sets
// kStatusCheck in *status on any violation; reads only within each series' own ranges.
cudaError_t launch_check_sort(const SeriesDesc *desc, int64_t S, const uint16_t *lab, const uint16_t *rk,
                              const int32_t *runs, int32_t *status, cudaStream_t st);
// crit (optional, may be null): the critical value of each reported change point.
cudaError_t launch_collect(const SeriesDesc *desc, int64_t S, const uint8_t *cp_flag, const int64_t *cp_num,
                           const int64_t *cp_den, const double *cp_p, const double *cp_crit, int32_t max_cp,
                           int32_t *cp_count, int32_t *cp_idx, int64_t *dnum, int64_t *dden, double *p, double *crit,
                           QueueHeader *q, cudaStream_t st);

// gate (optional): a device counter; when it reads 0 the proposal kernels return at once (a
// learned call whose every series the run sweep takes uses no proposal).
cudaError_t launch_summaries(const uint32_t *samples, const SeriesDesc *raw_desc, int64_t S, uint16_t *feat,
                             cudaStream_t st, const unsigned long long *gate = nullptr);

cudaError_t launch_latency_stats(const uint32_t *samples, const SeriesDesc *desc, int64_t S, double *mean_out,
                                 uint32_t *p50_out, uint32_t *p95_out, double *std_out, cudaStream_t st);
cudaError_t launch_reduce_rank(const uint32_t *samples, const SeriesDesc *raw_desc, int64_t S,
                               double *red, uint32_t *rank_out, cudaStream_t st);

}  // namespace mt4g
