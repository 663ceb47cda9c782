// C ABI of libmt4g: context, argument validation, workspace, and the call sequence
//   (reduce+rank for Eq. 2 mode) -> per-series radix sort + run table ->
//   (learned mode: features -> tensor-core network -> windows) ->
//   persistent work-queue kernel (scan, p-value, segmentation) -> collect,
// plus CUDA-graph replay, the scan-tile autotuner, the host-input pipeline that overlaps
// chunk copies with segmentation, the proposal network's training calls and measurement helpers.
#include <algorithm>
#include <map>
#include <cstdarg>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "mt4g_cnn.cuh"

using namespace mt4g;

struct mt4g_ctx {
    int device = 0;
    int grid = 0;        // CTAs of the slice-only queue kernel
    int grid_sweep = 0;  // CTAs of the queue kernel with the run sweep
    std::string err;
    long long wait_limit_ns = 5000000000LL;

    void *ws = nullptr;  // device workspace
    size_t ws_bytes = 0;
    void *pin = nullptr;  // pinned host staging for per-call tables
    size_t pin_bytes = 0;
    cudaEvent_t pin_free = nullptr;  // recorded after the last upload out of `pin`
    QueueHeader *h_hdr = nullptr;     // pinned: queue header (status, work) of the last call
    QueueHeader *hdr_dst = nullptr;   // when set, finish_call copies the header here instead
    // host-input segmentation (mt4g_ks_segment_host): two device staging buffers, a copy stream,
    // and the per-chunk queue headers that mt4g_wait() combines
    void *hin[2] = {nullptr, nullptr};
    size_t hin_bytes = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
    cudaStream_t up_stream = nullptr;  // while set: table uploads go on this stream (the copy stream)
    cudaEvent_t ev_up = nullptr;
    QueueHeader *h_chunk_hdr = nullptr;  // pinned
    int64_t chunk_hdr_cap = 0;
    int64_t n_chunk_hdr = 0;             // headers of the last host-input call, combined by mt4g_wait
    cudaStream_t last_stream = nullptr;
    bool have_last = false;      // some call has enqueued work on last_stream
    bool last_enqueued = false;  // the most recent call enqueued work (its status is in h_hdr)

    int32_t forced_kpt = 0;  // 0: per-series choice; 1, 2, 4: every series
    std::map<std::pair<int, int>, int32_t> tune;  // (floor log2 T, floor log2 m) -> scan tile
    int32_t n_win = 3;       // learned proposals: windows per series
    int32_t half = 16;       // window half width
    float conf_min = 0.9f;   // below: the series takes the plain scan
    float *learned_conf = nullptr;  // device: proposal confidence of the last learned call

    // proposal network
    CnnState cnn;
    bool cnn_alloc = false;
    bool cnn_ready = false;  // weights initialised or loaded
    void *cnn_ws = nullptr;  // activations, features, host-table copies
    size_t cnn_ws_bytes = 0;

    // stage timing: events of the last kTimingRing calls
    static constexpr int kTimingRing = 64;
    static constexpr int kMarks = 6;
    bool timing = false;
    bool events_made = false;
    cudaEvent_t ev[kTimingRing][kMarks] = {};
    int ring_pos = 0;
    int ring_count = 0;

    bool checks = false;  // MT4G_OPT_CHECKS: consistency check of the sort's output
    bool sweep_skip = false;  // MT4G_OPT_SWEEP_SKIP: exact bound skipping in the run sweep
    bool learned_windows = false;  // MT4G_OPT_LEARNED_WINDOWS: window-only scans of swept series

    // CUDA-graph replay of identical calls (MT4G_OPT_GRAPH)
    bool use_graph = false;
    bool capturing = false;       // inside a capture: no host syncs, staging from graph_pin
    void *graph_pin = nullptr;    // pinned staging owned by the captured graph
    size_t graph_pin_bytes = 0, graph_pin_off = 0;
    cudaGraphExec_t graph_exec = nullptr;
    uint64_t graph_key = 0;
    cudaStream_t graph_stream = nullptr;        // graphs are captured and launched here
    cudaEvent_t graph_in = nullptr, graph_out = nullptr;  // joins with the caller's stream
    long long cnn_version = 0;    // bumped whenever the weights change

    // work-queue ready flags carry an epoch so they need no clearing between calls
    uint32_t call_counter = 0;
    size_t ready_off = (size_t)-1;
    unsigned long long ready_cap = 0;
};

// NVTX range over an entry point's host-side work (header-only NVTX 3: free without a tool).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

namespace {

int fail(mt4g_ctx *c, int code, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
int fail(mt4g_ctx *c, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

#define CUDA_TRY(c, expr)                                                                                  \
    do {                                                                                                   \
        cudaError_t e_ = (expr);                                                                           \
        if (e_ != cudaSuccess)                                                                             \
            return fail((c), e_ == cudaErrorMemoryAllocation ? MT4G_ENOMEM : MT4G_ECUDA, "%s: %s (%s:%d)", \
                        #expr, cudaGetErrorString(e_), __FILE__, __LINE__);                                \
    } while (0)

// Bump allocator over the workspace: a layout pass computes the size, a second
// pass hands out pointers.
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base((char *)b) {}
    template <class T>
    T *take(size_t n) {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? (T *)(base + off) : nullptr;
        off += n * sizeof(T);
        return p;
    }
};

struct Plan {
    int64_t S = 0;
    int64_t Ntot = 0;    // samples fed to the sort (raw, or one per step in Eq. 2 mode)
    int64_t sumT = 0;
    bool reduced = false;
    int32_t min_seg = 1;
    std::vector<SeriesDesc> desc;      // sort/scan view
    std::vector<SeriesDesc> raw_desc;  // raw samples (Eq. 2 mode only)
    std::vector<int32_t> sort_order;   // series by size, largest first
    std::vector<int32_t> qorder;       // series by scan cost (T^2 m), costliest first
    std::vector<int64_t> item_base;    // first queue slot of the top-level slices of qorder[i]
    int64_t n_init = 0;                // top-level items
    int32_t top_parts = 1;             // parts of each top-level run-sweep segment
    unsigned long long cap = 0;
    bool learned = false;              // items are pushed by the learned init kernel
    bool use_sweep = false;            // run-sweep series present: ranks from the sort, sweep kernel
    unsigned long long rec_cap = 0;    // certification records (learned mode)
};

struct Buffers {
    QueueHeader *q;
    SeriesDesc *desc;
    SeriesDesc *raw_desc;
    int32_t *order;
    int32_t *qorder;
    int64_t *item_base;
    uint32_t *keyA, *keyB;
    uint16_t *labA, *labB;
    int32_t *runs;
    uint8_t *cp_flag;
    int64_t *cp_num, *cp_den;
    double *cp_p;
    double *cp_crit;
    WorkItem *items;
    int32_t *ready;
    uint32_t *gcount;
    CertRecord *recs;
    int32_t *fallback;
    double *red;
    uint32_t *rank;
};

size_t carve(void *base, const Plan &P, Buffers &B, size_t *ready_off) {
    Carver c(base);
    B.q = c.take<QueueHeader>(1);
    B.desc = c.take<SeriesDesc>(P.S);
    B.raw_desc = c.take<SeriesDesc>(P.reduced ? P.S : 0);
    B.order = c.take<int32_t>(P.S);
    B.qorder = c.take<int32_t>(P.S);
    B.item_base = c.take<int64_t>(P.S);
    B.keyA = c.take<uint32_t>(P.Ntot);
    B.keyB = c.take<uint32_t>(P.Ntot);
    B.labA = c.take<uint16_t>(P.Ntot);
    B.labB = c.take<uint16_t>(P.Ntot);
    B.runs = c.take<int32_t>(P.Ntot + P.S);
    B.cp_flag = c.take<uint8_t>(P.sumT);
    B.cp_num = c.take<int64_t>(P.sumT);
    B.cp_den = c.take<int64_t>(P.sumT);
    B.cp_p = c.take<double>(P.sumT);
    B.cp_crit = c.take<double>(P.sumT);
    B.red = c.take<double>(P.reduced ? P.sumT : 0);
    B.rank = c.take<uint32_t>(P.reduced ? P.sumT : 0);
    B.gcount = c.take<uint32_t>(P.cap);
    B.recs = c.take<CertRecord>(P.learned ? P.rec_cap : 0);
    B.fallback = c.take<int32_t>(P.S);
    B.items = c.take<WorkItem>(P.cap);
    B.ready = c.take<int32_t>(P.cap);
    *ready_off = (size_t)((char *)B.ready - (char *)base);
    return c.off + 256;
}

// Record stage boundary `i` of the current call when stage timing is on (not in graphs).
void mark(mt4g_ctx *ctx, int i, cudaStream_t st) {
    if (ctx->timing && !ctx->capturing) cudaEventRecord(ctx->ev[ctx->ring_pos][i], st);
}

// Scan tile for a series: split groups of 32 per warp work item.  A forced value
// (MT4G_OPT_SCAN_KPT) wins; otherwise the autotuned table, else a size heuristic.
int ilog2(int64_t v) {
    int b = 0;
    while (v > 1) {
        v >>= 1;
        b++;
    }
    return b;
}

constexpr int64_t kSweepLikelySamples = 1 << 17;

int32_t pick_kpt(const mt4g_ctx *ctx, int32_t T, int32_t m) {
    if (ctx->forced_kpt) return ctx->forced_kpt;
    const auto it = ctx->tune.find({ilog2(T), ilog2(m)});
    return it == ctx->tune.end() ? MT4G_SCAN_SWEEP : it->second;
}

// Validate the host tables and build the per-call plan.
int make_plan(mt4g_ctx *ctx, const int64_t *offsets, const int32_t *steps, int64_t S, int32_t mode,
              int32_t min_seg, Plan &P) {
    if (S < 0) return fail(ctx, MT4G_EINVAL, "S must be >= 0 (got %lld)", (long long)S);
    if (S > 0 && (!offsets || !steps)) return fail(ctx, MT4G_EINVAL, "offsets and steps must be non-NULL");
    if (S > (int64_t)INT32_MAX) return fail(ctx, MT4G_EINVAL, "too many series");
    if (mode != MT4G_MODE_FULL && mode != MT4G_MODE_REDUCED && mode != MT4G_MODE_LEARNED)
        return fail(ctx, MT4G_EINVAL, "mode must be MT4G_MODE_FULL, _REDUCED or _LEARNED (got %d)", mode);
    if (min_seg < 1) return fail(ctx, MT4G_EINVAL, "min_seg must be >= 1 (got %d)", min_seg);
    if (S > 0 && offsets[0] != 0) return fail(ctx, MT4G_EINVAL, "offsets[0] must be 0");
    P.S = S;
    P.reduced = mode == MT4G_MODE_REDUCED;
    P.min_seg = min_seg;
    P.desc.resize(S);
    if (P.reduced) P.raw_desc.resize(S);
    int64_t sumT = 0, ntot = 0;
    for (int64_t s = 0; s < S; s++) {
        const int64_t n = offsets[s + 1] - offsets[s];
        const int32_t T = steps[s];
        if (T < 2 || T > MT4G_MAX_STEPS)
            return fail(ctx, MT4G_EINVAL, "series %lld: T=%d outside [2, %d]", (long long)s, T, MT4G_MAX_STEPS);
        if (n <= 0 || n % T != 0)
            return fail(ctx, MT4G_EINVAL, "series %lld: %lld samples is not a positive multiple of T=%d",
                        (long long)s, (long long)n, T);
        if (n > MT4G_MAX_SERIES_SAMPLES)
            return fail(ctx, MT4G_EINVAL, "series %lld: %lld samples exceeds %lld", (long long)s, (long long)n,
                        (long long)MT4G_MAX_SERIES_SAMPLES);
        const int32_t m = (int32_t)(n / T);
        SeriesDesc d{};
        d.T = T;
        d.step_base = sumT;
        if (P.reduced) {
            SeriesDesc r{};
            r.off = offsets[s];
            r.T = T;
            r.m = m;
            r.step_base = sumT;
            P.raw_desc[s] = r;
            d.off = sumT;  // the ranks of the reduced values, one per step
            d.m = 1;
        } else {
            d.off = offsets[s];
            d.m = m;
        }
        d.run_base = d.off + s;
        const int32_t tile = pick_kpt(ctx, d.T, d.m);
        d.kpt = tile == MT4G_SCAN_SWEEP ? 0 : tile;
        P.desc[s] = d;
        sumT += T;
        ntot += (int64_t)d.T * d.m;
    }
    P.sumT = sumT;
    P.Ntot = ntot;
    // Run sweep or slices.  The sweep needs at most kSweepMaxRuns distinct values, which the
    // host cannot see before the sort; by default it is planned for series of at most
    // kSweepLikelySamples samples (a forced or tuned sweep is planned as asked), and taken
    // for the call when those series carry at least half of the estimated scan cost (T^2 m):
    // the sweep kernel holds fewer warps per SM, which would slow the slices of the others.
    // Series planned for the sweep that turn out to have more distinct values are scanned in
    // slices by that kernel.
    {
        const bool forced = ctx->forced_kpt != 0;
        double sw = 0.0, tot = 0.0;
        for (int64_t s = 0; s < S; s++) {
            SeriesDesc &d = P.desc[s];
            const double cost = (double)d.T * d.T * d.m;
            tot += cost;
            if (d.kpt != 0) continue;
            const bool tuned = ctx->tune.count({ilog2(d.T), ilog2(d.m)}) != 0;
            if (!forced && !tuned && (int64_t)d.T * d.m > kSweepLikelySamples)
                d.kpt = 1;
            else
                sw += cost;
        }
        P.use_sweep = sw > 0.0 && (ctx->forced_kpt == MT4G_SCAN_SWEEP || sw >= 0.5 * tot);
        if (!P.use_sweep)
            for (auto &d : P.desc)
                if (d.kpt == 0) d.kpt = 1;
    }
    // sort launch order: largest series first
    P.sort_order.resize(S);
    std::iota(P.sort_order.begin(), P.sort_order.end(), 0);
    bool uniform = true;
    for (int64_t s = 1; s < S && uniform; s++)
        uniform = P.desc[s].T == P.desc[0].T && P.desc[s].m == P.desc[0].m;
    if (!uniform) {
        std::stable_sort(P.sort_order.begin(), P.sort_order.end(), [&](int32_t a, int32_t b) {
            return (int64_t)P.desc[a].T * P.desc[a].m > (int64_t)P.desc[b].T * P.desc[b].m;
        });
    }
    // first work items: the top-level slices, costliest series (T^2 m) first
    P.qorder = P.sort_order;
    if (!uniform) {
        std::stable_sort(P.qorder.begin(), P.qorder.end(), [&](int32_t a, int32_t b) {
            const double ca = (double)P.desc[a].T * P.desc[a].T * P.desc[a].m;
            const double cb = (double)P.desc[b].T * P.desc[b].T * P.desc[b].m;
            return ca > cb;
        });
    }
    // top-level run-sweep segments are cut into parts when the launch has more warps than
    // such series (a small batch), so that no warp starts idle
    int64_t n_sweep = 0;
    for (const auto &d : P.desc) n_sweep += d.kpt == 0;
    if (n_sweep > 0) {
        const int64_t warps = (int64_t)ctx->grid_sweep * (kSweepThreads / 32);
        P.top_parts = (int32_t)std::max<int64_t>(1, std::min<int64_t>(kSweepMaxParts, warps / n_sweep));
    }
    P.item_base.resize(S);
    int64_t nb = 0;
    for (int64_t i = 0; i < S; i++) {
        P.item_base[i] = nb;
        const SeriesDesc &d = P.desc[P.qorder[i]];
        nb += d.kpt == 0 ? sweep_parts(d.T, min_seg, P.top_parts) : seg_chunks(d.T, min_seg, d.kpt);
    }
    P.n_init = nb;
    // slices of the children of accepted splits: a split of a segment adds at most
    // two slices beyond the parent's, so 2 per step plus the top level bounds them
    // for the usual few change points per series; overflow is reported.
    P.cap = (unsigned long long)nb + 4ull * (unsigned long long)sumT + 1024ull;
    P.learned = mode == MT4G_MODE_LEARNED;
    if (P.learned) {
        // probe groups (windows + grid) and refinements come on top of the plain slices
        P.cap += 8ull * (unsigned long long)S + 2ull * (unsigned long long)sumT;
        P.rec_cap = 16ull * (unsigned long long)S + 1024ull;
    }
    return MT4G_OK;
}

int ensure_workspace(mt4g_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->ws_bytes) return MT4G_OK;
    if (ctx->capturing) return fail(ctx, MT4G_ECUDA, "workspace growth during graph capture");
    if (ctx->have_last) CUDA_TRY(ctx, cudaStreamSynchronize(ctx->last_stream));
    if (ctx->graph_exec) {  // the captured graph points into the old workspace
        cudaGraphExecDestroy(ctx->graph_exec);
        ctx->graph_exec = nullptr;
    }
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    ctx->ready_off = (size_t)-1;
    const size_t want = bytes + bytes / 8;
    CUDA_TRY(ctx, cudaMalloc(&ctx->ws, want));
    ctx->ws_bytes = want;
    return MT4G_OK;
}

int ensure_pinned(mt4g_ctx *ctx, size_t bytes) {
    if (ctx->capturing) return fail(ctx, MT4G_ECUDA, "pinned staging during graph capture");
    CUDA_TRY(ctx, cudaEventSynchronize(ctx->pin_free));
    if (bytes <= ctx->pin_bytes) return MT4G_OK;
    if (ctx->pin) cudaFreeHost(ctx->pin);
    ctx->pin = nullptr;
    ctx->pin_bytes = 0;
    const size_t want = bytes + bytes / 4 + 4096;
    CUDA_TRY(ctx, cudaMallocHost(&ctx->pin, want));
    ctx->pin_bytes = want;
    return MT4G_OK;
}

// Host staging for uploads: the context's pinned buffer (after the previous uploads out of
// it completed), or, while a graph is being captured, a slice of the graph's own buffer
// (its contents must stay valid for every replay).
unsigned char *stage_alloc(mt4g_ctx *ctx, size_t bytes, int *rc) {
    *rc = MT4G_OK;
    if (ctx->capturing) {
        const size_t at = (ctx->graph_pin_off + 255) & ~(size_t)255;
        if (at + bytes > ctx->graph_pin_bytes) {
            *rc = fail(ctx, MT4G_ECUDA, "graph staging buffer too small");
            return nullptr;
        }
        ctx->graph_pin_off = at + bytes;
        return (unsigned char *)ctx->graph_pin + at;
    }
    *rc = ensure_pinned(ctx, bytes);
    return *rc ? nullptr : (unsigned char *)ctx->pin;
}

cudaError_t staged(mt4g_ctx *ctx, cudaStream_t st) {
    return ctx->capturing ? cudaSuccess : cudaEventRecord(ctx->pin_free, st);
}

// A call's host-to-device table uploads go on the call's stream, except during a host-input
// call: there they go on its copy stream, queued in order with the chunk copies, because every
// H2D copy of the device shares one copy engine and an upload behind the next chunk's copy would
// hold up the current chunk.  uploads_done makes the call's stream wait for them.
cudaStream_t upload_stream(const mt4g_ctx *ctx, cudaStream_t st) { return ctx->up_stream ? ctx->up_stream : st; }

cudaError_t uploads_done(mt4g_ctx *ctx, cudaStream_t us, cudaStream_t st) {
    if (us == st) return cudaSuccess;
    cudaError_t e = cudaEventRecord(ctx->ev_up, us);
    return e != cudaSuccess ? e : cudaStreamWaitEvent(st, ctx->ev_up, 0);
}

// Everything a call enqueues up to (and including) the work-queue kernel.
int enqueue_pipeline(mt4g_ctx *ctx, const uint32_t *samples, Plan &P, RunParams &R, Buffers &B, cudaStream_t st) {
    size_t ready_off = 0;
    const size_t need = carve(nullptr, P, B, &ready_off);
    int rc = ensure_workspace(ctx, need);
    if (rc) return rc;
    carve(ctx->ws, P, B, &ready_off);

    // epoch of this call's ready flags; clear them when the layout changed or the epoch wraps.
    // A captured graph clears them on every replay and uses a fixed epoch.
    uint32_t e = 0x7fff;
    bool fresh = true;
    if (!ctx->capturing) {
        ctx->call_counter++;
        e = ctx->call_counter & 0x7fff;
        fresh = ready_off != ctx->ready_off || P.cap > ctx->ready_cap || e == 0;
        if (e == 0) {
            ctx->call_counter++;
            e = ctx->call_counter & 0x7fff;
        }
    }
    const uint32_t epoch = e << 16;
    if (fresh) {
        CUDA_TRY(ctx, cudaMemsetAsync(B.ready, 0, P.cap * sizeof(int32_t), st));
        ctx->ready_off = ready_off;
        ctx->ready_cap = P.cap;
    }

    // stage the host tables in pinned memory and upload them
    const size_t n_items = (size_t)P.n_init;
    const size_t bytes_hdr = sizeof(QueueHeader);
    const size_t bytes_desc = P.S * sizeof(SeriesDesc);
    const size_t bytes_raw = P.reduced ? P.S * sizeof(SeriesDesc) : 0;
    const size_t bytes_order = P.S * sizeof(int32_t);
    const size_t bytes_items = P.S * sizeof(int32_t);   // qorder
    const size_t bytes_ready = P.S * sizeof(int64_t);   // item_base
    char *h = (char *)stage_alloc(ctx, bytes_hdr + bytes_desc + bytes_raw + bytes_order + bytes_items + bytes_ready + 64,
                                  &rc);
    if (rc) return rc;
    QueueHeader hq{};
    hq.head = 0;
    hq.tail = P.learned ? 0 : n_items;
    hq.pending = P.learned ? 0 : (long long)n_items;
    hq.status = 0;
    hq.cap = P.cap;
    hq.rec_cap = P.rec_cap;
    size_t o = 0;
    memcpy(h + o, &hq, bytes_hdr);
    o += bytes_hdr;
    memcpy(h + o, P.desc.data(), bytes_desc);
    const size_t o_desc = o;
    o += bytes_desc;
    const size_t o_raw = o;
    if (bytes_raw) memcpy(h + o, P.raw_desc.data(), bytes_raw);
    o += bytes_raw;
    const size_t o_order = o;
    memcpy(h + o, P.sort_order.data(), bytes_order);
    o += bytes_order;
    const size_t o_items = o;
    if (bytes_items) memcpy(h + o, P.qorder.data(), bytes_items);
    o += bytes_items;
    o = (o + 7) & ~(size_t)7;
    const size_t o_ready = o;
    if (bytes_ready) memcpy(h + o, P.item_base.data(), bytes_ready);

    const cudaStream_t us = upload_stream(ctx, st);
    CUDA_TRY(ctx, cudaMemcpyAsync(B.q, h, bytes_hdr, cudaMemcpyHostToDevice, us));
    if (bytes_desc) CUDA_TRY(ctx, cudaMemcpyAsync(B.desc, h + o_desc, bytes_desc, cudaMemcpyHostToDevice, us));
    if (bytes_raw) CUDA_TRY(ctx, cudaMemcpyAsync(B.raw_desc, h + o_raw, bytes_raw, cudaMemcpyHostToDevice, us));
    if (bytes_order) CUDA_TRY(ctx, cudaMemcpyAsync(B.order, h + o_order, bytes_order, cudaMemcpyHostToDevice, us));
    if (bytes_items) CUDA_TRY(ctx, cudaMemcpyAsync(B.qorder, h + o_items, bytes_items, cudaMemcpyHostToDevice, us));
    if (bytes_ready)
        CUDA_TRY(ctx, cudaMemcpyAsync(B.item_base, h + o_ready, bytes_ready, cudaMemcpyHostToDevice, us));
    CUDA_TRY(ctx, staged(ctx, us));
    CUDA_TRY(ctx, uploads_done(ctx, us, st));
    if (!P.learned)
        CUDA_TRY(ctx, launch_init_items(B.desc, B.qorder, B.item_base, P.S, P.min_seg, P.top_parts, B.items,
                                        B.ready, B.gcount, epoch, st));
    mark(ctx, 1, st);

    const uint32_t *sort_in = samples;
    if (P.reduced) {
        CUDA_TRY(ctx, launch_reduce_rank(samples, B.raw_desc, P.S, B.red, B.rank, st));
        sort_in = B.rank;
    }
    CUDA_TRY(ctx, launch_sort(sort_in, B.desc, B.order, P.S, B.keyA, B.keyB, B.labA, B.labB, B.runs,
                              P.use_sweep ? &B.q->ranked : nullptr, st));
    if (ctx->checks) CUDA_TRY(ctx, launch_check_sort(B.desc, P.S, B.labA, B.labB, B.runs, &B.q->status, st));
    mark(ctx, 2, st);

    R = RunParams{};
    R.desc = B.desc;
    R.lab = B.labA;
    R.rk = P.use_sweep ? B.labB : nullptr;
    R.runs = B.runs;
    R.q = B.q;
    R.items = B.items;
    R.ready = B.ready;
    R.gcount = B.gcount;
    R.recs = B.recs;
    R.fallback = B.fallback;
    R.min_seg = P.min_seg;
    R.wait_limit_ns = ctx->wait_limit_ns;
    R.cp_flag = B.cp_flag;
    R.cp_num = B.cp_num;
    R.cp_den = B.cp_den;
    R.cp_p = B.cp_p;
    R.cp_crit = B.cp_crit;
    R.sweep_warps = ctx->grid_sweep * (kSweepThreads / 32);
    R.sweep_skip = ctx->sweep_skip ? 1 : 0;
    R.top_parts = P.top_parts;
    return (int)epoch;  // >= 0
}

int enqueue_proposals(mt4g_ctx *ctx, const uint32_t *samples, Plan &P, Buffers &B, RunParams &R, cudaStream_t st);

int finish_call(mt4g_ctx *ctx, Buffers &B, cudaStream_t st) {
    mark(ctx, 5, st);
    if (ctx->timing && !ctx->capturing) {
        ctx->ring_pos = (ctx->ring_pos + 1) % mt4g_ctx::kTimingRing;
        ctx->ring_count = std::min(ctx->ring_count + 1, mt4g_ctx::kTimingRing);
    }
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->hdr_dst ? ctx->hdr_dst : ctx->h_hdr, B.q, sizeof(QueueHeader),
                                  cudaMemcpyDeviceToHost, st));
    ctx->last_stream = st;
    ctx->have_last = true;
    ctx->last_enqueued = true;
    return MT4G_OK;
}

int begin_call(mt4g_ctx *ctx) {
    if (!ctx) return MT4G_EINVAL;
    ctx->err.clear();
    ctx->last_enqueued = false;
    ctx->n_chunk_hdr = 0;
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    return MT4G_OK;
}

}  // namespace

extern "C" {

int mt4g_create(mt4g_ctx **out, int device) {
    if (!out) return MT4G_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return MT4G_ECUDA;
    mt4g_ctx *c = new (std::nothrow) mt4g_ctx();
    if (!c) return MT4G_ENOMEM;
    c->device = device;
    if (cudaSetDevice(device) != cudaSuccess || cudaEventCreateWithFlags(&c->pin_free, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&c->h_hdr, sizeof(QueueHeader)) != cudaSuccess) {
        delete c;
        return MT4G_ECUDA;
    }
    memset(c->h_hdr, 0, sizeof(QueueHeader));
    c->grid = queue_grid(device);
    c->grid_sweep = queue_grid_sweep(device);
    if (c->grid <= 0 || c->grid_sweep <= 0) {
        delete c;
        return MT4G_ECUDA;
    }
    *out = c;
    return MT4G_OK;
}

void mt4g_destroy(mt4g_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->have_last) cudaStreamSynchronize(c->last_stream);
    if (c->pin_free) {
        cudaEventSynchronize(c->pin_free);
        cudaEventDestroy(c->pin_free);
    }
    if (c->ws) cudaFree(c->ws);
    if (c->cnn_ws) cudaFree(c->cnn_ws);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph_pin) cudaFreeHost(c->graph_pin);
    if (c->graph_stream) {
        cudaStreamSynchronize(c->graph_stream);
        cudaStreamDestroy(c->graph_stream);
        cudaEventDestroy(c->graph_in);
        cudaEventDestroy(c->graph_out);
    }
    if (c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        cudaStreamDestroy(c->copy_stream);
        for (int b = 0; b < 2; b++) {
            cudaEventDestroy(c->ev_copied[b]);
            cudaEventDestroy(c->ev_free[b]);
        }
        cudaEventDestroy(c->ev_up);
    }
    for (int b = 0; b < 2; b++)
        if (c->hin[b]) cudaFree(c->hin[b]);
    if (c->h_chunk_hdr) cudaFreeHost(c->h_chunk_hdr);
    if (c->cnn_alloc) cudaFree(c->cnn.master);
    if (c->pin) cudaFreeHost(c->pin);
    if (c->h_hdr) cudaFreeHost(c->h_hdr);
    if (c->events_made)
        for (auto &row : c->ev)
            for (auto &e : row) cudaEventDestroy(e);
    delete c;
}

const char *mt4g_last_error(const mt4g_ctx *c) { return c ? c->err.c_str() : "no context"; }

int mt4g_set_option(mt4g_ctx *c, int option, int64_t value) {
    if (!c) return MT4G_EINVAL;
    if (option == MT4G_OPT_STAGE_TIMING) {
        if (value && !c->events_made) {
            CUDA_TRY(c, cudaSetDevice(c->device));
            for (auto &row : c->ev)
                for (auto &e : row) CUDA_TRY(c, cudaEventCreate(&e));
            c->events_made = true;
        }
        c->timing = value != 0;
        c->ring_pos = 0;
        c->ring_count = 0;
        return MT4G_OK;
    }
    if (option == MT4G_OPT_SCAN_KPT) {
        if (value != 0 && value != 1 && value != 2 && value != 4 && value != MT4G_SCAN_SWEEP)
            return fail(c, MT4G_EINVAL, "scan tile must be 0 (automatic), 1, 2, 4 or %d (run sweep)",
                        MT4G_SCAN_SWEEP);
        c->forced_kpt = (int32_t)value;
        return MT4G_OK;
    }
    if (option == MT4G_OPT_GRAPH) {
        c->use_graph = value != 0;
        return MT4G_OK;
    }
    if (option == MT4G_OPT_CHECKS) {
        c->checks = value != 0;
        return MT4G_OK;
    }
    if (option == MT4G_OPT_SWEEP_SKIP) {
        c->sweep_skip = value != 0;
        return MT4G_OK;
    }
    if (option == MT4G_OPT_LEARNED_WINDOWS) {
        c->learned_windows = value != 0;
        return MT4G_OK;
    }
    if (option == MT4G_OPT_WINDOWS) {
        if (value < 1 || value > 8) return fail(c, MT4G_EINVAL, "windows must be 1..8");
        c->n_win = (int32_t)value;
        return MT4G_OK;
    }
    if (option == MT4G_OPT_HALF_WIDTH) {
        if (value < 0 || value > 31) return fail(c, MT4G_EINVAL, "half width must be 0..31");
        c->half = (int32_t)value;
        return MT4G_OK;
    }
    if (option == MT4G_OPT_CONF_MIN_PPM) {
        if (value < 0 || value > 1000001) return fail(c, MT4G_EINVAL, "confidence threshold must be 0..1000001 ppm");
        c->conf_min = (float)((double)value * 1e-6);
        return MT4G_OK;
    }
    if (option == MT4G_OPT_WAIT_LIMIT_NS) {
        if (value <= 0) return fail(c, MT4G_EINVAL, "wait limit must be > 0 ns");
        c->wait_limit_ns = value;
        return MT4G_OK;
    }
    return fail(c, MT4G_EINVAL, "unknown option %d", option);
}

int mt4g_wait(mt4g_ctx *c) {
    if (!c) return MT4G_EINVAL;
    if (!c->have_last) return MT4G_OK;
    CUDA_TRY(c, cudaSetDevice(c->device));
    CUDA_TRY(c, cudaStreamSynchronize(c->last_stream));
    if (!c->last_enqueued) return MT4G_OK;
    if (c->n_chunk_hdr > 0) {  // a host-input call: combine its chunks' headers
        QueueHeader sum{};
        for (int64_t i = 0; i < c->n_chunk_hdr; i++) {
            const QueueHeader &h = c->h_chunk_hdr[i];
            sum.status |= h.status;
            sum.evals += h.evals;
            sum.certified += h.certified;
            sum.refined += h.refined;
            sum.rec_next += h.rec_next;
            sum.swept += h.swept;
            sum.ranked += h.ranked;
            sum.counted += h.counted;
            sum.unswept += h.unswept;
        }
        *c->h_hdr = sum;
        c->n_chunk_hdr = 0;
    }
    const int32_t st = c->h_hdr->status;
    if (st & kStatusCheck) return fail(c, MT4G_ECHECK, "device consistency check of the sort output failed");
    if (st & kStatusTimeout) return fail(c, MT4G_ETIMEOUT, "a bounded device-side wait expired");
    if (st & kStatusQueueFull) return fail(c, MT4G_ECAPACITY, "work queue capacity exceeded");
    if (st & kStatusCapacity) return fail(c, MT4G_ECAPACITY, "a series has more than max_cp change points");
    return MT4G_OK;
}

static int scan_body(mt4g_ctx *ctx, const uint32_t *samples, const int64_t *offsets, const int32_t *steps,
                     int64_t S, int32_t mode, int32_t *k_out, int64_t *dnum_out, int64_t *dden_out, double *p_out,
                     void *cuda_stream) {
    int rc = MT4G_OK;
    if (S > 0 && (!samples || !k_out || !dnum_out || !dden_out || !p_out))
        return fail(ctx, MT4G_EINVAL, "NULL device pointer");
    Plan P;
    rc = make_plan(ctx, offsets, steps, S, mode, 1, P);
    if (rc) return rc;
    if (S == 0) return MT4G_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    Buffers B;
    RunParams R;
    mark(ctx, 0, st);
    const int epoch = enqueue_pipeline(ctx, samples, P, R, B, st);
    if (epoch < 0) return epoch;
    R.mode = kRunScan;
    R.k_out = k_out;
    R.dnum_out = dnum_out;
    R.dden_out = dden_out;
    R.p_out = p_out;
    mark(ctx, 3, st);
    CUDA_TRY(ctx, launch_queue_run(R, R.rk ? ctx->grid_sweep : ctx->grid, (uint32_t)epoch, st));
    mark(ctx, 4, st);
    return finish_call(ctx, B, st);
}

static int segment_body(mt4g_ctx *ctx, const uint32_t *samples, const int64_t *offsets, const int32_t *steps,
                        int64_t S, double alpha, int32_t min_seg, int32_t max_cp, int32_t mode, int32_t *cp_count,
                        int32_t *cp_idx, int64_t *dnum, int64_t *dden, double *p, int32_t *fallback, double *crit,
                        void *cuda_stream) {
    int rc = MT4G_OK;
    if (!(alpha > 0.0 && alpha < 1.0)) return fail(ctx, MT4G_EINVAL, "alpha must be in (0, 1)");
    if (max_cp < 0) return fail(ctx, MT4G_EINVAL, "max_cp must be >= 0");
    if (S > 0 && (!samples || !cp_count || (max_cp > 0 && (!cp_idx || !dnum || !dden || !p))))
        return fail(ctx, MT4G_EINVAL, "NULL device pointer");
    if (mode == MT4G_MODE_LEARNED && !ctx->cnn_ready)
        return fail(ctx, MT4G_EINVAL, "learned mode needs weights: call mt4g_cnn_load or mt4g_cnn_init");
    Plan P;
    rc = make_plan(ctx, offsets, steps, S, mode, min_seg, P);
    if (rc) return rc;
    if (mode == MT4G_MODE_LEARNED)
        for (int64_t s = 0; s < S; s++)
            if (P.desc[s].m > 256)
                return fail(ctx, MT4G_EINVAL, "series %lld: learned mode needs m <= 256", (long long)s);
    if (S == 0) return MT4G_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    Buffers B;
    RunParams R;
    mark(ctx, 0, st);
    const int epoch = enqueue_pipeline(ctx, samples, P, R, B, st);
    if (epoch < 0) return epoch;
    R.mode = P.learned ? kRunLearned : kRunSegment;
    R.win_only = P.learned && ctx->learned_windows && R.rk ? 1 : 0;
    R.alpha = alpha;
    // Eq. 1's constant -1/2 ln(alpha / 2), once on the host; each accepted split multiplies it
    // by (n_L + n_R) / (n_L n_R) (critical value beside the change point)
    R.crit_c = -0.5 * log(alpha / 2.0);
    CUDA_TRY(ctx, cudaMemsetAsync(B.cp_flag, 0, (size_t)P.sumT, st));
    if (P.learned) {
        rc = enqueue_proposals(ctx, samples, P, B, R, st);
        if (rc) return rc;
        mark(ctx, 3, st);
        CUDA_TRY(ctx, launch_init_learned(R, ctx->learned_conf, ctx->conf_min, B.fallback, P.S, (uint32_t)epoch, st));
    } else {
        CUDA_TRY(ctx, cudaMemsetAsync(B.fallback, 0, P.S * sizeof(int32_t), st));
    }
    if (!P.learned) mark(ctx, 3, st);
    CUDA_TRY(ctx, launch_queue_run(R, R.rk ? ctx->grid_sweep : ctx->grid, (uint32_t)epoch, st));
    mark(ctx, 4, st);
    CUDA_TRY(ctx, launch_collect(B.desc, P.S, B.cp_flag, B.cp_num, B.cp_den, B.cp_p, B.cp_crit, max_cp, cp_count,
                                 cp_idx, dnum, dden, p, crit, B.q, st));
    if (fallback)
        CUDA_TRY(ctx, cudaMemcpyAsync(fallback, B.fallback, P.S * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    return finish_call(ctx, B, st);
}


}  // extern "C"

namespace {

uint64_t fnv1a(uint64_t h, const void *p, size_t n) {
    const unsigned char *b = (const unsigned char *)p;
    for (size_t i = 0; i < n; i++) h = (h ^ b[i]) * 0x100000001b3ULL;
    return h;
}

template <class T>
uint64_t fnv_val(uint64_t h, const T &v) {
    return fnv1a(h, &v, sizeof(T));
}

// Run `body` directly, or (MT4G_OPT_GRAPH) as one CUDA-graph launch: a call identical to
// the captured one (same key) replays it; otherwise `presize` grows every buffer first,
// then the call is captured with no host synchronisation inside and launched.
template <class Presize, class Body>
int run_maybe_graph(mt4g_ctx *ctx, uint64_t key, size_t pin_bytes, cudaStream_t user_st, Presize &&presize,
                    Body &&body) {
    if (!ctx->use_graph) return body(user_st);
    // the caller's stream may be the legacy default stream, which cannot be captured: capture
    // and launch on the context's own stream, ordered after and before the caller's work
    if (!ctx->graph_stream) {
        CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->graph_stream, cudaStreamNonBlocking));
        CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->graph_in, cudaEventDisableTiming));
        CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->graph_out, cudaEventDisableTiming));
    }
    cudaStream_t st = ctx->graph_stream;
    CUDA_TRY(ctx, cudaEventRecord(ctx->graph_in, user_st));
    CUDA_TRY(ctx, cudaStreamWaitEvent(st, ctx->graph_in, 0));
    if (ctx->graph_exec && ctx->graph_key == key) {
        CUDA_TRY(ctx, cudaGraphLaunch(ctx->graph_exec, st));
    } else {
        if (ctx->have_last) CUDA_TRY(ctx, cudaStreamSynchronize(ctx->last_stream));
        if (ctx->graph_exec) {
            cudaGraphExecDestroy(ctx->graph_exec);
            ctx->graph_exec = nullptr;
        }
        int rc = presize();
        if (rc) return rc;
        if (pin_bytes > ctx->graph_pin_bytes) {
            if (ctx->graph_pin) cudaFreeHost(ctx->graph_pin);
            ctx->graph_pin = nullptr;
            ctx->graph_pin_bytes = 0;
            CUDA_TRY(ctx, cudaMallocHost(&ctx->graph_pin, pin_bytes));
            ctx->graph_pin_bytes = pin_bytes;
        }
        ctx->graph_pin_off = 0;
        CUDA_TRY(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        ctx->capturing = true;
        rc = body(st);
        ctx->capturing = false;
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(st, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return fail(ctx, MT4G_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
        const cudaError_t ei = cudaGraphInstantiate(&ctx->graph_exec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            ctx->graph_exec = nullptr;
            return fail(ctx, MT4G_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ei));
        }
        ctx->graph_key = key;
        CUDA_TRY(ctx, cudaGraphLaunch(ctx->graph_exec, st));
    }
    CUDA_TRY(ctx, cudaEventRecord(ctx->graph_out, st));
    CUDA_TRY(ctx, cudaStreamWaitEvent(user_st, ctx->graph_out, 0));
    ctx->ready_off = (size_t)-1;  // a later direct call clears the flags the graph used
    ctx->last_stream = user_st;
    ctx->have_last = true;
    ctx->last_enqueued = true;
    return MT4G_OK;
}

uint64_t call_key(const mt4g_ctx *ctx, int entry, const void *samples, const int64_t *offsets, const int32_t *steps,
                  int64_t S, int32_t mode, double alpha, int32_t min_seg, int32_t max_cp, const void *const *outs,
                  int n_outs, void *stream) {
    uint64_t h = 0xcbf29ce484222325ULL;
    h = fnv_val(h, entry);
    h = fnv_val(h, samples);
    h = fnv_val(h, S);
    h = fnv_val(h, mode);
    h = fnv_val(h, alpha);
    h = fnv_val(h, min_seg);
    h = fnv_val(h, max_cp);
    h = fnv_val(h, stream);
    h = fnv_val(h, ctx->n_win);
    h = fnv_val(h, ctx->half);
    h = fnv_val(h, ctx->conf_min);
    h = fnv_val(h, ctx->forced_kpt);
    h = fnv_val(h, ctx->checks);
    h = fnv_val(h, ctx->sweep_skip);
    h = fnv_val(h, ctx->learned_windows);
    h = fnv_val(h, ctx->cnn_version);
    for (int i = 0; i < n_outs; i++) h = fnv_val(h, outs[i]);
    if (S > 0 && offsets && steps) {
        h = fnv1a(h, offsets, (size_t)(S + 1) * sizeof(int64_t));
        h = fnv1a(h, steps, (size_t)S * sizeof(int32_t));
    }
    return h;
}

size_t graph_pin_need(int64_t S) { return (size_t)S * 256 + 8192; }

int presize_cnn(mt4g_ctx *ctx, int64_t rows, int64_t S);  // proposal workspace (defined below)

int presize_for(mt4g_ctx *ctx, const int64_t *offsets, const int32_t *steps, int64_t S, int32_t mode,
                int32_t min_seg) {
    if (S <= 0) return MT4G_OK;
    Plan P;
    int rc = make_plan(ctx, offsets, steps, S, mode, min_seg, P);
    if (rc) return rc;
    Buffers B;
    size_t ready_off = 0;
    rc = ensure_workspace(ctx, carve(nullptr, P, B, &ready_off));
    if (rc) return rc;
    if (mode == MT4G_MODE_LEARNED) rc = presize_cnn(ctx, P.sumT + 4 * S, S);
    return rc;
}

}  // namespace

extern "C" {

int mt4g_ks_scan(mt4g_ctx *ctx, const uint32_t *samples, const int64_t *offsets, const int32_t *steps, int64_t S,
                 int32_t mode, int32_t *k_out, int64_t *dnum_out, int64_t *dden_out, double *p_out,
                 void *cuda_stream) {
    NvtxRange nvtx("mt4g_ks_scan");
    int rc = begin_call(ctx);
    if (rc) return rc;
    if (mode == MT4G_MODE_LEARNED) return fail(ctx, MT4G_EINVAL, "mt4g_ks_scan has no learned mode");
    const void *outs[4] = {k_out, dnum_out, dden_out, p_out};
    const uint64_t key = ctx->use_graph ? call_key(ctx, 1, samples, offsets, steps, S, mode, 0.0, 1, 0, outs, 4,
                                                   cuda_stream)
                                        : 0;
    return run_maybe_graph(
        ctx, key, graph_pin_need(S), (cudaStream_t)cuda_stream,
        [&] { return presize_for(ctx, offsets, steps, S, mode, 1); },
        [&](cudaStream_t s) {
            return scan_body(ctx, samples, offsets, steps, S, mode, k_out, dnum_out, dden_out, p_out, (void *)s);
        });
}

int mt4g_ks_segment(mt4g_ctx *ctx, const uint32_t *samples, const int64_t *offsets, const int32_t *steps, int64_t S,
                    double alpha, int32_t min_seg, int32_t max_cp, int32_t mode, int32_t *cp_count, int32_t *cp_idx,
                    int64_t *dnum, int64_t *dden, double *p, int32_t *fallback, double *crit, void *cuda_stream) {
    NvtxRange nvtx("mt4g_ks_segment");
    int rc = begin_call(ctx);
    if (rc) return rc;
    const void *outs[7] = {cp_count, cp_idx, dnum, dden, p, fallback, crit};
    const uint64_t key = ctx->use_graph ? call_key(ctx, 2, samples, offsets, steps, S, mode, alpha, min_seg, max_cp,
                                                   outs, 7, cuda_stream)
                                        : 0;
    return run_maybe_graph(
        ctx, key, graph_pin_need(S), (cudaStream_t)cuda_stream,
        [&] { return presize_for(ctx, offsets, steps, S, mode, min_seg); },
        [&](cudaStream_t s) {
            return segment_body(ctx, samples, offsets, steps, S, alpha, min_seg, max_cp, mode, cp_count, cp_idx, dnum,
                                dden, p, fallback, crit, (void *)s);
        });
}

int mt4g_ks_segment_host(mt4g_ctx *ctx, const uint32_t *samples_host, const int64_t *offsets, const int32_t *steps,
                         int64_t S, double alpha, int32_t min_seg, int32_t max_cp, int32_t mode,
                         int64_t chunk_samples, int32_t *cp_count, int32_t *cp_idx, int64_t *dnum, int64_t *dden,
                         double *p, int32_t *fallback, double *crit, void *cuda_stream) {
    NvtxRange nvtx("mt4g_ks_segment_host");
    int rc = begin_call(ctx);
    if (rc) return rc;
    if (S < 0 || (S > 0 && (!offsets || !steps))) return fail(ctx, MT4G_EINVAL, "bad host tables");
    if (S == 0) return MT4G_OK;
    if (!samples_host) return fail(ctx, MT4G_EINVAL, "NULL host sample pointer");
    if (offsets[0] != 0) return fail(ctx, MT4G_EINVAL, "offsets[0] must be 0");
    // everything a chunk's segmentation would reject, checked before any chunk is enqueued
    if (!(alpha > 0.0 && alpha < 1.0)) return fail(ctx, MT4G_EINVAL, "alpha must be in (0, 1)");
    if (max_cp < 0) return fail(ctx, MT4G_EINVAL, "max_cp must be >= 0");
    if (min_seg < 1) return fail(ctx, MT4G_EINVAL, "min_seg must be >= 1 (got %d)", min_seg);
    if (mode != MT4G_MODE_FULL && mode != MT4G_MODE_REDUCED && mode != MT4G_MODE_LEARNED)
        return fail(ctx, MT4G_EINVAL, "mode must be MT4G_MODE_FULL, _REDUCED or _LEARNED (got %d)", mode);
    if (mode == MT4G_MODE_LEARNED && !ctx->cnn_ready)
        return fail(ctx, MT4G_EINVAL, "learned mode needs weights: call mt4g_cnn_load or mt4g_cnn_init");
    if (!cp_count || (max_cp > 0 && (!cp_idx || !dnum || !dden || !p)))
        return fail(ctx, MT4G_EINVAL, "NULL device pointer");
    for (int64_t s = 0; s < S; s++) {
        const int64_t n = offsets[s + 1] - offsets[s];
        const int32_t T = steps[s];
        if (T < 2 || T > MT4G_MAX_STEPS)
            return fail(ctx, MT4G_EINVAL, "series %lld: T=%d outside [2, %d]", (long long)s, T, MT4G_MAX_STEPS);
        if (n <= 0 || n % T != 0 || n > MT4G_MAX_SERIES_SAMPLES)
            return fail(ctx, MT4G_EINVAL, "series %lld: %lld samples is not a positive multiple of T=%d within %lld",
                        (long long)s, (long long)n, T, (long long)MT4G_MAX_SERIES_SAMPLES);
        if (mode == MT4G_MODE_LEARNED && n / T > 256)
            return fail(ctx, MT4G_EINVAL, "series %lld: learned mode needs m <= 256", (long long)s);
    }
    // default: about eight chunks (the first copy and the last chunk's work are not overlapped;
    // much smaller chunks leave the GPU underused), none below 2^24 samples
    if (chunk_samples <= 0) chunk_samples = std::max<int64_t>((int64_t)1 << 24, (offsets[S] + 7) / 8);
    // chunks: consecutive series up to chunk_samples samples (a larger series is a chunk alone)
    std::vector<int64_t> first{0};
    for (int64_t s = 1; s < S; s++)
        if (offsets[s + 1] - offsets[first.back()] > chunk_samples) first.push_back(s);
    first.push_back(S);
    const int64_t nchunks = (int64_t)first.size() - 1;
    int64_t max_chunk = 0;
    for (int64_t c = 0; c < nchunks; c++) max_chunk = std::max(max_chunk, offsets[first[c + 1]] - offsets[first[c]]);
    const size_t need = (size_t)max_chunk * sizeof(uint32_t);
    // staging buffers, copy stream, events, per-chunk headers (grown on demand)
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (need > ctx->hin_bytes) {
        CUDA_TRY(ctx, cudaDeviceSynchronize());
        for (int b = 0; b < 2; b++) {
            if (ctx->hin[b]) cudaFree(ctx->hin[b]);
            ctx->hin[b] = nullptr;
        }
        ctx->hin_bytes = 0;
        for (int b = 0; b < 2; b++)
            if (cudaMalloc(&ctx->hin[b], need) != cudaSuccess)
                return fail(ctx, MT4G_ENOMEM, "cannot allocate %zu bytes of input staging", need);
        ctx->hin_bytes = need;
    }
    if (!ctx->copy_stream) {
        CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
        for (int b = 0; b < 2; b++) {
            CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->ev_copied[b], cudaEventDisableTiming));
            CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->ev_free[b], cudaEventDisableTiming));
        }
        CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->ev_up, cudaEventDisableTiming));
    }
    if (nchunks > ctx->chunk_hdr_cap) {
        if (ctx->have_last) CUDA_TRY(ctx, cudaStreamSynchronize(ctx->last_stream));
        if (ctx->h_chunk_hdr) cudaFreeHost(ctx->h_chunk_hdr);
        ctx->h_chunk_hdr = nullptr;
        ctx->chunk_hdr_cap = 0;
        if (cudaMallocHost(&ctx->h_chunk_hdr, (size_t)nchunks * sizeof(QueueHeader)) != cudaSuccess)
            return fail(ctx, MT4G_ENOMEM, "cannot allocate pinned chunk headers");
        ctx->chunk_hdr_cap = nchunks;
    }
    // the previous user of the staging buffers must be done with them
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->copy_stream));
    if (ctx->have_last && ctx->last_stream != st) CUDA_TRY(ctx, cudaStreamSynchronize(ctx->last_stream));
    for (int b = 0; b < 2; b++) CUDA_TRY(ctx, cudaEventRecord(ctx->ev_free[b], st));
    std::vector<int64_t> loc;
    for (int64_t c = 0; c < nchunks; c++) {
        NvtxRange chunk_range("mt4g_ks_segment_host chunk");
        const int b = (int)(c & 1);
        const int64_t s0 = first[c], n = first[c + 1] - first[c];
        const int64_t base = offsets[s0], cnt = offsets[first[c + 1]] - base;
        // copy chunk c while chunk c - 1 is processed; buffer b is free once chunk c - 2 is done
        CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_free[b], 0));
        CUDA_TRY(ctx, cudaMemcpyAsync(ctx->hin[b], samples_host + base, (size_t)cnt * sizeof(uint32_t),
                                      cudaMemcpyHostToDevice, ctx->copy_stream));
        CUDA_TRY(ctx, cudaEventRecord(ctx->ev_copied[b], ctx->copy_stream));
        CUDA_TRY(ctx, cudaStreamWaitEvent(st, ctx->ev_copied[b], 0));
        loc.assign(offsets + s0, offsets + s0 + n + 1);
        for (auto &o : loc) o -= base;
        // the chunk's table uploads (on the copy stream, after this copy) overwrite the context's
        // workspace: the previous chunk must be done with it
        if (c > 0) CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_free[b ^ 1], 0));
        ctx->hdr_dst = ctx->h_chunk_hdr + c;
        ctx->up_stream = ctx->copy_stream;
        rc = segment_body(ctx, (const uint32_t *)ctx->hin[b], loc.data(), steps + s0, n, alpha, min_seg, max_cp, mode,
                          cp_count + s0, max_cp ? cp_idx + s0 * max_cp : cp_idx, max_cp ? dnum + s0 * max_cp : dnum,
                          max_cp ? dden + s0 * max_cp : dden, max_cp ? p + s0 * max_cp : p,
                          fallback ? fallback + s0 : nullptr, (crit && max_cp) ? crit + s0 * max_cp : nullptr,
                          (void *)st);
        ctx->hdr_dst = nullptr;
        ctx->up_stream = nullptr;
        if (rc) return rc;
        CUDA_TRY(ctx, cudaEventRecord(ctx->ev_free[b], st));
    }
    ctx->n_chunk_hdr = nchunks;
    ctx->last_enqueued = true;
    return MT4G_OK;
}

int mt4g_stage_times(mt4g_ctx *c, double *ms_out, int32_t max_calls) {
    if (!c || (max_calls > 0 && !ms_out)) return MT4G_EINVAL;
    if (!c->timing) return fail(c, MT4G_EINVAL, "stage timing is off (MT4G_OPT_STAGE_TIMING)");
    const int n = std::min<int>(max_calls, c->ring_count);
    CUDA_TRY(c, cudaSetDevice(c->device));
    for (int i = 0; i < n; i++) {
        const int slot = (c->ring_pos - n + i + mt4g_ctx::kTimingRing) % mt4g_ctx::kTimingRing;
        CUDA_TRY(c, cudaEventSynchronize(c->ev[slot][mt4g_ctx::kMarks - 1]));
        for (int j = 0; j + 1 < mt4g_ctx::kMarks; j++) {
            float ms = 0.f;
            CUDA_TRY(c, cudaEventElapsedTime(&ms, c->ev[slot][j], c->ev[slot][j + 1]));
            ms_out[i * (mt4g_ctx::kMarks - 1) + j] = ms;
        }
    }
    return n;
}

int mt4g_last_work(mt4g_ctx *c, int64_t *evals) {
    if (!c || !evals) return MT4G_EINVAL;
    *evals = (int64_t)c->h_hdr->evals;
    return MT4G_OK;
}

}  // extern "C"

// ====================================================================== proposal network

namespace {

int ensure_cnn_state(mt4g_ctx *c) {
    if (c->cnn_alloc) return MT4G_OK;
    float *base = nullptr;
    const size_t n = (size_t)kCnnParams;
    // master, used, flipped (2 x 5120), m1, m2, grad, loss, then FP64 gradients
    const size_t nf = 6 * n + 2 * 5120 + 64;
    CUDA_TRY(c, cudaMalloc(&base, nf * sizeof(float) + n * sizeof(double) + 256));
    CnnState &W = c->cnn;
    W.master = base;
    W.used = base + n;
    W.m1 = base + 2 * n;
    W.m2 = base + 3 * n;
    W.grad = base + 4 * n;
    W.flipped = base + 5 * n;
    W.loss = base + 5 * n + 2 * 5120;
    W.grad64 = (double *)(((uintptr_t)(base + nf) + 255) & ~(uintptr_t)255);
    CUDA_TRY(c, cudaMemset(base, 0, nf * sizeof(float)));
    c->cnn_alloc = true;
    return MT4G_OK;
}

struct CnnBuffers {
    CnnActs A;
    uint16_t *feat;
    SeriesDesc *desc;
    int64_t *tiles_before;  // tiles of 128 positions (training passes)
    int64_t *infer_before;  // tiles of the one-kernel inference
    int64_t ninfer;
    int32_t *win;
    float *conf;
};

// Layout of the proposal workspace for `rows` padded rows and S series.
size_t carve_cnn(void *base, int64_t rows, int64_t S, bool training, bool own_feat, int32_t n_win, CnnBuffers &B) {
    Carver c(base);
    // hidden activations in memory only for the backward pass; inference keeps them on chip
    B.A.a1 = c.take<uint16_t>(training ? rows * 32 : 0);
    B.A.a2 = c.take<uint16_t>(training ? rows * 32 : 0);
    B.A.a3 = c.take<uint16_t>(training ? rows * 32 : 0);
    B.A.logits = c.take<float>(rows);
    B.A.g = c.take<float>(training ? rows : 0);
    B.A.dz1 = c.take<float>(training ? rows * 32 : 0);
    B.A.dz2 = c.take<float>(training ? rows * 32 : 0);
    B.A.dz3 = c.take<float>(training ? rows * 32 : 0);
    B.A.inv_valid = c.take<float>(16);
    B.tiles_before = c.take<int64_t>(2 * S);  // the two tile prefixes, uploaded together
    B.A.tiles_before = B.tiles_before;
    B.infer_before = B.tiles_before ? B.tiles_before + S : nullptr;
    B.desc = c.take<SeriesDesc>(S);
    B.feat = c.take<uint16_t>(own_feat ? rows * kFeatC : 0);
    B.win = c.take<int32_t>(own_feat ? S * n_win : 0);
    B.conf = c.take<float>(own_feat ? S : 0);
    return c.off + 256;
}

int ensure_cnn_ws(mt4g_ctx *c, size_t bytes) {
    if (bytes <= c->cnn_ws_bytes) return MT4G_OK;
    if (c->capturing) return fail(c, MT4G_ECUDA, "workspace growth during graph capture");
    if (c->have_last) CUDA_TRY(c, cudaStreamSynchronize(c->last_stream));
    if (c->graph_stream) CUDA_TRY(c, cudaStreamSynchronize(c->graph_stream));
    if (c->graph_exec) {  // the captured graph points into the old workspace; its stream,
        cudaGraphExecDestroy(c->graph_exec);  // events and pinned staging stay for the next capture
        c->graph_exec = nullptr;
    }
    if (c->cnn_ws) cudaFree(c->cnn_ws);
    c->cnn_ws = nullptr;
    c->cnn_ws_bytes = 0;
    const size_t want = bytes + bytes / 8;
    CUDA_TRY(c, cudaMalloc(&c->cnn_ws, want));
    c->cnn_ws_bytes = want;
    return MT4G_OK;
}

// Host tables of a feature batch: descriptors (step bases) and tile prefixes.
int upload_cnn_tables(mt4g_ctx *c, const std::vector<SeriesDesc> &desc, CnnBuffers &B, int64_t *ntiles,
                      cudaStream_t st) {
    std::vector<int64_t> tb, ib;
    *ntiles = cnn_tiles(desc, tb);
    B.ninfer = cnn_infer_tiles(desc, ib);
    const size_t S = desc.size();
    int rc = MT4G_OK;
    char *h = (char *)stage_alloc(c, S * (sizeof(SeriesDesc) + 2 * sizeof(int64_t)) + 64, &rc);
    if (rc) return rc;
    memcpy(h, desc.data(), S * sizeof(SeriesDesc));
    memcpy(h + S * sizeof(SeriesDesc), tb.data(), S * sizeof(int64_t));
    memcpy(h + S * (sizeof(SeriesDesc) + sizeof(int64_t)), ib.data(), S * sizeof(int64_t));
    const cudaStream_t us = upload_stream(c, st);
    CUDA_TRY(c, cudaMemcpyAsync(B.desc, h, S * sizeof(SeriesDesc), cudaMemcpyHostToDevice, us));
    CUDA_TRY(c, cudaMemcpyAsync(B.tiles_before, h + S * sizeof(SeriesDesc), 2 * S * sizeof(int64_t),
                                cudaMemcpyHostToDevice, us));
    CUDA_TRY(c, staged(c, us));
    CUDA_TRY(c, uploads_done(c, us, st));
    return MT4G_OK;
}

// Zero pad rows of the training pass's activation and gradient arrays.
int zero_pads(mt4g_ctx *c, CnnBuffers &B, int64_t S, cudaStream_t st) {
    CUDA_TRY(c, launch_zero_pad_rows(B.A.a1, 64, B.desc, S, st));
    CUDA_TRY(c, launch_zero_pad_rows(B.A.a2, 64, B.desc, S, st));
    CUDA_TRY(c, launch_zero_pad_rows(B.A.a3, 64, B.desc, S, st));
    CUDA_TRY(c, launch_zero_pad_rows(B.A.g, 4, B.desc, S, st));
    CUDA_TRY(c, launch_zero_pad_rows(B.A.dz1, 128, B.desc, S, st));
    CUDA_TRY(c, launch_zero_pad_rows(B.A.dz2, 128, B.desc, S, st));
    CUDA_TRY(c, launch_zero_pad_rows(B.A.dz3, 128, B.desc, S, st));
    return MT4G_OK;
}

std::vector<SeriesDesc> feature_desc(const int32_t *steps, int64_t S) {
    std::vector<SeriesDesc> d(S);
    int64_t sb = 0;
    for (int64_t s = 0; s < S; s++) {
        d[s] = SeriesDesc{};
        d[s].T = steps[s];
        d[s].m = 1;
        d[s].step_base = sb;
        sb += steps[s];
    }
    return d;
}

int check_steps(mt4g_ctx *c, const int32_t *steps, int64_t S) {
    if (S < 0 || (S > 0 && !steps)) return fail(c, MT4G_EINVAL, "bad steps table");
    for (int64_t s = 0; s < S; s++)
        if (steps[s] < 2 || steps[s] > MT4G_MAX_STEPS) return fail(c, MT4G_EINVAL, "series %lld: bad T", (long long)s);
    return MT4G_OK;
}

// He-uniform initial weights from splitmix64(seed, index); zero biases.
void init_weights_host(uint64_t seed, std::vector<float> &w) {
    w.assign(kCnnParams, 0.f);
    const int cins[4] = {17, 32, 32, 32}, cinp[4] = {kFeatC, 32, 32, 32}, couts[4] = {32, 32, 32, 1};
    uint64_t x = seed * 0x9E3779B97F4A7C15ULL + 0x632BE59BD9B4E019ULL;
    for (int l = 0; l < 4; l++) {
        const float bound = sqrtf(6.f / (float)(cins[l] * 5));
        const int off = cnn_off(2 * l);
        for (int dd = 0; dd < 5; dd++)
            for (int i = 0; i < cinp[l]; i++)
                for (int o = 0; o < couts[l]; o++) {
                    uint64_t z = (x += 0x9E3779B97F4A7C15ULL);
                    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
                    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
                    z ^= z >> 31;
                    const float u = (float)((z >> 40) * 0x1.0p-24);  // [0, 1)
                    w[off + (dd * cinp[l] + i) * couts[l] + o] = i < cins[l] ? (2.f * u - 1.f) * bound : 0.f;
                }
    }
}

uint32_t crc32_update(uint32_t crc, const void *data, size_t n) {
    const uint8_t *p = (const uint8_t *)data;
    crc = ~crc;
    for (size_t i = 0; i < n; i++) {
        crc ^= p[i];
        for (int k = 0; k < 8; k++) crc = (crc >> 1) ^ (0xEDB88320u & (0u - (crc & 1u)));
    }
    return ~crc;
}

struct CnnFileHeader {
    char magic[8];  // "MT4GCNN1"
    int32_t n_params;
    int32_t feat_channels;
    int64_t adam_step;
    uint32_t crc;  // CRC-32 of the three arrays that follow
    uint32_t pad;
};

}  // namespace

extern "C" {

int mt4g_cnn_init(mt4g_ctx *c, uint64_t seed) {
    int rc = begin_call(c);
    if (rc) return rc;
    c->cnn_version++;
    rc = ensure_cnn_state(c);
    if (rc) return rc;
    std::vector<float> w;
    init_weights_host(seed, w);
    CUDA_TRY(c, cudaMemcpy(c->cnn.master, w.data(), kCnnParams * sizeof(float), cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemset(c->cnn.m1, 0, kCnnParams * sizeof(float)));
    CUDA_TRY(c, cudaMemset(c->cnn.m2, 0, kCnnParams * sizeof(float)));
    c->cnn.step = 0;
    c->cnn_ready = true;
    return MT4G_OK;
}

int mt4g_cnn_get_params(mt4g_ctx *c, float *host_out) {
    int rc = begin_call(c);
    if (rc) return rc;
    if (!c->cnn_ready) return fail(c, MT4G_EINVAL, "no weights: call mt4g_cnn_init or mt4g_cnn_load");
    if (!host_out) return fail(c, MT4G_EINVAL, "NULL output");
    if (c->have_last) CUDA_TRY(c, cudaStreamSynchronize(c->last_stream));
    CUDA_TRY(c, cudaMemcpy(host_out, c->cnn.master, kCnnParams * sizeof(float), cudaMemcpyDeviceToHost));
    return MT4G_OK;
}

int mt4g_cnn_set_params(mt4g_ctx *c, const float *host_in) {
    int rc = begin_call(c);
    if (rc) return rc;
    c->cnn_version++;
    if (!host_in) return fail(c, MT4G_EINVAL, "NULL input");
    rc = ensure_cnn_state(c);
    if (rc) return rc;
    if (c->have_last) CUDA_TRY(c, cudaStreamSynchronize(c->last_stream));
    CUDA_TRY(c, cudaMemcpy(c->cnn.master, host_in, kCnnParams * sizeof(float), cudaMemcpyHostToDevice));
    c->cnn_ready = true;
    return MT4G_OK;
}

int mt4g_cnn_save(mt4g_ctx *c, const char *path) {
    int rc = begin_call(c);
    if (rc) return rc;
    if (!c->cnn_ready) return fail(c, MT4G_EINVAL, "no weights to save");
    if (!path) return fail(c, MT4G_EINVAL, "NULL path");
    if (c->have_last) CUDA_TRY(c, cudaStreamSynchronize(c->last_stream));
    std::vector<float> buf(3 * (size_t)kCnnParams);
    CUDA_TRY(c, cudaMemcpy(buf.data(), c->cnn.master, kCnnParams * sizeof(float), cudaMemcpyDeviceToHost));
    CUDA_TRY(c, cudaMemcpy(buf.data() + kCnnParams, c->cnn.m1, kCnnParams * sizeof(float), cudaMemcpyDeviceToHost));
    CUDA_TRY(c, cudaMemcpy(buf.data() + 2 * kCnnParams, c->cnn.m2, kCnnParams * sizeof(float),
                           cudaMemcpyDeviceToHost));
    CnnFileHeader h{};
    memcpy(h.magic, "MT4GCNN1", 8);
    h.n_params = kCnnParams;
    h.feat_channels = kFeatC;
    h.adam_step = c->cnn.step;
    h.crc = crc32_update(0, buf.data(), buf.size() * sizeof(float));
    FILE *f = fopen(path, "wb");
    if (!f) return fail(c, MT4G_EINVAL, "cannot open %s for writing", path);
    const bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    fclose(f);
    return ok ? MT4G_OK : fail(c, MT4G_EINVAL, "short write to %s", path);
}

int mt4g_cnn_load(mt4g_ctx *c, const char *path) {
    int rc = begin_call(c);
    if (rc) return rc;
    c->cnn_version++;
    if (!path) return fail(c, MT4G_EINVAL, "NULL path");
    FILE *f = fopen(path, "rb");
    if (!f) return fail(c, MT4G_EINVAL, "cannot open %s", path);
    CnnFileHeader h{};
    std::vector<float> buf(3 * (size_t)kCnnParams);
    const bool ok = fread(&h, sizeof(h), 1, f) == 1 && fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    fclose(f);
    if (!ok || memcmp(h.magic, "MT4GCNN1", 8) != 0 || h.n_params != kCnnParams || h.feat_channels != kFeatC)
        return fail(c, MT4G_EINVAL, "%s is not a weights file of this network", path);
    if (crc32_update(0, buf.data(), buf.size() * sizeof(float)) != h.crc)
        return fail(c, MT4G_EINVAL, "%s: checksum mismatch", path);
    rc = ensure_cnn_state(c);
    if (rc) return rc;
    if (c->have_last) CUDA_TRY(c, cudaStreamSynchronize(c->last_stream));
    CUDA_TRY(c, cudaMemcpy(c->cnn.master, buf.data(), kCnnParams * sizeof(float), cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemcpy(c->cnn.m1, buf.data() + kCnnParams, kCnnParams * sizeof(float), cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemcpy(c->cnn.m2, buf.data() + 2 * kCnnParams, kCnnParams * sizeof(float),
                           cudaMemcpyHostToDevice));
    c->cnn.step = h.adam_step;
    c->cnn_ready = true;
    return MT4G_OK;
}

int mt4g_summaries(mt4g_ctx *ctx, const uint32_t *samples, const int64_t *offsets, const int32_t *steps, int64_t S,
                   uint16_t *feat_out, void *cuda_stream) {
    NvtxRange nvtx("mt4g_summaries");
    int rc = begin_call(ctx);
    if (rc) return rc;
    if (S > 0 && (!samples || !feat_out)) return fail(ctx, MT4G_EINVAL, "NULL device pointer");
    Plan P;
    rc = make_plan(ctx, offsets, steps, S, MT4G_MODE_FULL, 1, P);
    if (rc) return rc;
    for (int64_t s = 0; s < S; s++)
        if (P.desc[s].m > 256) return fail(ctx, MT4G_EINVAL, "series %lld: summaries need m <= 256", (long long)s);
    if (S == 0) return MT4G_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    Buffers B;
    RunParams R;
    mark(ctx, 0, st);
    const int epoch = enqueue_pipeline(ctx, samples, P, R, B, st);
    if (epoch < 0) return epoch;
    CUDA_TRY(ctx, launch_summaries(samples, B.desc, S, feat_out, st));
    mark(ctx, 3, st);
    mark(ctx, 4, st);
    return finish_call(ctx, B, st);
}

int mt4g_latency_stats(mt4g_ctx *ctx, const uint32_t *samples, const int64_t *offsets, const int32_t *steps,
                       int64_t S, double *mean_out, uint32_t *p50_out, uint32_t *p95_out, double *std_out,
                       void *cuda_stream) {
    NvtxRange nvtx("mt4g_latency_stats");
    int rc = begin_call(ctx);
    if (rc) return rc;
    if (S > 0 && (!samples || !mean_out || !p50_out || !p95_out || !std_out))
        return fail(ctx, MT4G_EINVAL, "NULL device pointer");
    Plan P;
    rc = make_plan(ctx, offsets, steps, S, MT4G_MODE_FULL, 1, P);
    if (rc) return rc;
    if (S == 0) return MT4G_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    Buffers B;
    RunParams R;
    mark(ctx, 0, st);
    const int epoch = enqueue_pipeline(ctx, samples, P, R, B, st);
    if (epoch < 0) return epoch;
    mark(ctx, 3, st);
    CUDA_TRY(ctx, launch_latency_stats(samples, B.desc, S, mean_out, p50_out, p95_out, std_out, st));
    mark(ctx, 4, st);
    return finish_call(ctx, B, st);
}

int mt4g_cnn_forward(mt4g_ctx *c, const uint16_t *feat, const int32_t *steps, int64_t S, float *logits_out,
                     void *cuda_stream) {
    NvtxRange nvtx("mt4g_cnn_forward");
    int rc = begin_call(c);
    if (rc) return rc;
    if (!c->cnn_ready) return fail(c, MT4G_EINVAL, "no weights: call mt4g_cnn_init or mt4g_cnn_load");
    rc = check_steps(c, steps, S);
    if (rc) return rc;
    if (S == 0) return MT4G_OK;
    if (!feat || !logits_out) return fail(c, MT4G_EINVAL, "NULL device pointer");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    std::vector<SeriesDesc> desc = feature_desc(steps, S);
    const int64_t rows = desc.back().step_base + desc.back().T + 4 * S;
    CnnBuffers B;
    const size_t need = carve_cnn(nullptr, rows, S, false, false, 0, B);
    rc = ensure_cnn_ws(c, need);
    if (rc) return rc;
    carve_cnn(c->cnn_ws, rows, S, false, false, 0, B);
    B.A.logits = logits_out;
    int64_t ntiles = 0;
    rc = upload_cnn_tables(c, desc, B, &ntiles, st);
    if (rc) return rc;
    CUDA_TRY(c, cnn_prepare(c->cnn, st));
    CUDA_TRY(c, cnn_infer(c->cnn, feat, logits_out, B.desc, B.infer_before, S, B.ninfer, c->wait_limit_ns, nullptr,
                          st));
    c->last_stream = st;
    c->have_last = true;
    return MT4G_OK;
}

// Forward + backward on a batch of B series with T steps each (features in the padded
// layout); gradients into grad_out (device, kCnnParams) or the context's scratch.
static int cnn_fwd_bwd(mt4g_ctx *c, const uint16_t *feat, int32_t T, int64_t Bn, const int32_t *cp_count,
                       const int32_t *cp_idx, int32_t max_cp, float *grad_out, float *loss_out, cudaStream_t st) {
    if (!c->cnn_ready) return fail(c, MT4G_EINVAL, "no weights: call mt4g_cnn_init or mt4g_cnn_load");
    if (T < 2 || T > MT4G_MAX_STEPS || Bn < 1 || max_cp < 1 || !feat || !cp_count || !cp_idx)
        return fail(c, MT4G_EINVAL, "bad training batch arguments");
    std::vector<int32_t> steps(Bn, T);
    std::vector<SeriesDesc> desc = feature_desc(steps.data(), Bn);
    const int64_t rows = Bn * (int64_t)(T + 4);
    CnnBuffers B;
    const size_t need = carve_cnn(nullptr, rows, Bn, true, false, 0, B);
    int rc = ensure_cnn_ws(c, need);
    if (rc) return rc;
    carve_cnn(c->cnn_ws, rows, Bn, true, false, 0, B);
    int64_t ntiles = 0;
    rc = upload_cnn_tables(c, desc, B, &ntiles, st);
    if (rc) return rc;
    rc = zero_pads(c, B, Bn, st);
    if (rc) return rc;
    CUDA_TRY(c, cnn_prepare(c->cnn, st));
    CUDA_TRY(c, cnn_forward(c->cnn, feat, B.A, B.desc, B.tiles_before, Bn, ntiles, c->wait_limit_ns, nullptr, st));
    CUDA_TRY(c, cnn_backward(c->cnn, feat, B.A, cp_count, cp_idx, max_cp, B.desc, Bn, T, grad_out,
                             loss_out ? loss_out : c->cnn.loss, st));
    c->last_stream = st;
    c->have_last = true;
    return MT4G_OK;
}

int mt4g_cnn_grads(mt4g_ctx *c, const uint16_t *feat, int32_t T, int64_t B, const int32_t *cp_count,
                   const int32_t *cp_idx, int32_t max_cp, float *grad_out, float *loss_out, void *cuda_stream) {
    NvtxRange nvtx("mt4g_cnn_grads");
    int rc = begin_call(c);
    if (rc) return rc;
    if (!grad_out) return fail(c, MT4G_EINVAL, "NULL gradient buffer");
    return cnn_fwd_bwd(c, feat, T, B, cp_count, cp_idx, max_cp, grad_out, loss_out, (cudaStream_t)cuda_stream);
}

int mt4g_cnn_train_step(mt4g_ctx *c, const uint16_t *feat, int32_t T, int64_t B, const int32_t *cp_count,
                        const int32_t *cp_idx, int32_t max_cp, float lr, float *loss_out, void *cuda_stream) {
    NvtxRange nvtx("mt4g_cnn_train_step");
    int rc = begin_call(c);
    if (rc) return rc;
    if (!(lr > 0.f)) return fail(c, MT4G_EINVAL, "learning rate must be > 0");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    rc = cnn_fwd_bwd(c, feat, T, B, cp_count, cp_idx, max_cp, c->cnn.grad, loss_out, st);
    if (rc) return rc;
    c->cnn_version++;
    CUDA_TRY(c, cnn_adam(c->cnn, c->cnn.grad, lr, st));
    return MT4G_OK;
}

int mt4g_propose(mt4g_ctx *ctx, const uint32_t *samples, const int64_t *offsets, const int32_t *steps, int64_t S,
                 int32_t n_win, int32_t half_width, int32_t *win_center, float *conf, void *cuda_stream) {
    NvtxRange nvtx("mt4g_propose");
    int rc = begin_call(ctx);
    if (rc) return rc;
    if (!ctx->cnn_ready) return fail(ctx, MT4G_EINVAL, "no weights: call mt4g_cnn_init or mt4g_cnn_load");
    if (n_win < 1 || n_win > 8 || half_width < 0) return fail(ctx, MT4G_EINVAL, "need 1 <= n_win <= 8, half >= 0");
    if (S > 0 && (!samples || !win_center || !conf)) return fail(ctx, MT4G_EINVAL, "NULL device pointer");
    Plan P;
    rc = make_plan(ctx, offsets, steps, S, MT4G_MODE_FULL, 1, P);
    if (rc) return rc;
    for (int64_t s = 0; s < S; s++)
        if (P.desc[s].m > 256) return fail(ctx, MT4G_EINVAL, "series %lld: proposals need m <= 256", (long long)s);
    if (S == 0) return MT4G_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    Buffers B;
    RunParams R;
    mark(ctx, 0, st);
    const int epoch = enqueue_pipeline(ctx, samples, P, R, B, st);
    if (epoch < 0) return epoch;
    const int64_t rows = P.sumT + 4 * S;
    CnnBuffers C;
    const size_t need = carve_cnn(nullptr, rows, S, false, true, n_win, C);
    rc = ensure_cnn_ws(ctx, need);
    if (rc) return rc;
    carve_cnn(ctx->cnn_ws, rows, S, false, true, n_win, C);
    int64_t ntiles = 0;
    rc = upload_cnn_tables(ctx, P.desc, C, &ntiles, st);
    if (rc) return rc;
    CUDA_TRY(ctx, launch_summaries(samples, B.desc, S, C.feat, st));
    CUDA_TRY(ctx, cnn_prepare(ctx->cnn, st));
    CUDA_TRY(ctx, cnn_infer(ctx->cnn, C.feat, C.A.logits, B.desc, C.infer_before, S, C.ninfer, ctx->wait_limit_ns,
                            &B.q->status, st));
    CUDA_TRY(ctx, launch_propose(C.A.logits, B.desc, S, n_win, half_width, win_center, conf, st));
    mark(ctx, 3, st);
    mark(ctx, 4, st);
    return finish_call(ctx, B, st);
}

}  // extern "C"

namespace {

int presize_cnn(mt4g_ctx *ctx, int64_t rows, int64_t S) {
    CnnBuffers C;
    return ensure_cnn_ws(ctx, carve_cnn(nullptr, rows, S, false, true, ctx->n_win, C));
}

// Learned mode: features, logits and windows of every series (after the sort has written
// the medians), for the learned init kernel and the probe groups.
int enqueue_proposals(mt4g_ctx *ctx, const uint32_t *samples, Plan &P, Buffers &B, RunParams &R, cudaStream_t st) {
    const int64_t S = P.S;
    const int64_t rows = P.sumT + 4 * S;
    CnnBuffers C;
    const size_t need = carve_cnn(nullptr, rows, S, false, true, ctx->n_win, C);
    int rc = ensure_cnn_ws(ctx, need);
    if (rc) return rc;
    carve_cnn(ctx->cnn_ws, rows, S, false, true, ctx->n_win, C);
    int64_t ntiles = 0;
    rc = upload_cnn_tables(ctx, P.desc, C, &ntiles, st);
    if (rc) return rc;
    // in sweep calls the sort counted the series the sweep does not take: only they use the
    // proposals (unless swept series are scanned in their windows), and with none the proposal
    // kernels return at once
    const unsigned long long *gate = P.use_sweep && !ctx->learned_windows ? &B.q->unswept : nullptr;
    CUDA_TRY(ctx, launch_summaries(samples, B.desc, S, C.feat, st, gate));
    CUDA_TRY(ctx, cnn_prepare(ctx->cnn, st));
    CUDA_TRY(ctx, cnn_infer(ctx->cnn, C.feat, C.A.logits, B.desc, C.infer_before, S, C.ninfer, ctx->wait_limit_ns,
                            &B.q->status, st, gate));
    CUDA_TRY(ctx, launch_propose(C.A.logits, B.desc, S, ctx->n_win, ctx->half, C.win, C.conf, st, gate));
    R.win_center = C.win;
    R.n_win = ctx->n_win;
    R.half = ctx->half;
    ctx->learned_conf = C.conf;
    return MT4G_OK;
}

}  // namespace

extern "C" int mt4g_learned_stats(mt4g_ctx *c, int64_t *out) {
    if (!c || !out) return MT4G_EINVAL;
    out[0] = (int64_t)c->h_hdr->certified;
    out[1] = (int64_t)c->h_hdr->refined;
    out[2] = (int64_t)c->h_hdr->rec_next;
    return MT4G_OK;
}


extern "C" int mt4g_last_sweep(mt4g_ctx *c, int64_t *out) {
    if (!c || !out) return MT4G_EINVAL;
    out[0] = (int64_t)c->h_hdr->swept;
    out[1] = (int64_t)c->h_hdr->ranked;
    out[2] = (int64_t)c->h_hdr->counted;
    out[3] = (int64_t)c->h_hdr->unswept;
    return MT4G_OK;
}

extern "C" int mt4g_selftest_wait_timeout(mt4g_ctx *ctx, int64_t limit_ns, void *cuda_stream) {
    int rc = begin_call(ctx);
    if (rc) return rc;
    if (limit_ns <= 0 || limit_ns > 2000000000LL) return fail(ctx, MT4G_EINVAL, "limit must be in (0, 2e9] ns");
    // a one-series plan only to size the workspace; the queue header then claims one pending
    // item that is never published, so every warp's bounded wait expires
    const int64_t offsets[2] = {0, 2};
    const int32_t steps[1] = {2};
    Plan P;
    rc = make_plan(ctx, offsets, steps, 1, MT4G_MODE_FULL, 1, P);
    if (rc) return rc;
    size_t ready_off = 0;
    Buffers B;
    const size_t need = carve(nullptr, P, B, &ready_off);
    rc = ensure_workspace(ctx, need);
    if (rc) return rc;
    carve(ctx->ws, P, B, &ready_off);
    ctx->ready_off = (size_t)-1;  // the flags are cleared below; force a clear on the next call too
    cudaStream_t st = (cudaStream_t)cuda_stream;
    rc = ensure_pinned(ctx, sizeof(QueueHeader));
    if (rc) return rc;
    QueueHeader hq{};
    hq.pending = 1;
    hq.tail = 0;
    hq.cap = P.cap;
    memcpy(ctx->pin, &hq, sizeof(hq));
    CUDA_TRY(ctx, cudaMemcpyAsync(B.q, ctx->pin, sizeof(hq), cudaMemcpyHostToDevice, st));
    CUDA_TRY(ctx, cudaEventRecord(ctx->pin_free, st));
    CUDA_TRY(ctx, cudaMemsetAsync(B.ready, 0, P.cap * sizeof(int32_t), st));
    RunParams R{};
    R.desc = B.desc;
    R.lab = B.labA;
    R.runs = B.runs;
    R.q = B.q;
    R.items = B.items;
    R.ready = B.ready;
    R.gcount = B.gcount;
    R.mode = kRunScan;
    R.min_seg = 1;
    R.wait_limit_ns = limit_ns;
    CUDA_TRY(ctx, launch_queue_run(R, ctx->grid, 1u << 16, st));
    return finish_call(ctx, B, st);
}

extern "C" double mt4g_critical_value(double alpha, int64_t n_left, int64_t n_right) {
    if (!(alpha > 0.0 && alpha < 1.0) || n_left < 1 || n_right < 1) return -1.0;
    return sqrt(-0.5 * log(alpha / 2.0) * (double)(n_left + n_right) / ((double)n_left * (double)n_right));
}


extern "C" int mt4g_autotune(mt4g_ctx *ctx, const uint32_t *samples, const int64_t *offsets, const int32_t *steps,
                             int64_t S, void *cuda_stream) {
    int rc = begin_call(ctx);
    if (rc) return rc;
    Plan P;
    rc = make_plan(ctx, offsets, steps, S, MT4G_MODE_FULL, 1, P);
    if (rc) return rc;
    if (S == 0) return MT4G_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    CUDA_TRY(ctx, cudaStreamSynchronize(st));
    std::map<std::pair<int, int>, std::vector<int64_t>> buckets;
    for (int64_t s = 0; s < S; s++) {
        auto &v = buckets[{ilog2(P.desc[s].T), ilog2(P.desc[s].m)}];
        if (v.size() < 256) v.push_back(s);
    }
    const bool was_graph = ctx->use_graph, was_timing = ctx->timing;
    const int32_t was_forced = ctx->forced_kpt;
    ctx->use_graph = false;
    ctx->timing = false;
    uint32_t *gather = nullptr;
    int32_t *ko = nullptr;
    int64_t *no = nullptr, *dn = nullptr;
    double *po = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    rc = MT4G_OK;
    for (auto &kv : buckets) {
        const std::vector<int64_t> &ids = kv.second;
        const int64_t n = (int64_t)ids.size();
        std::vector<int64_t> offs(n + 1, 0);
        std::vector<int32_t> stp(n);
        for (int64_t i = 0; i < n; i++) {
            stp[i] = steps[ids[i]];
            offs[i + 1] = offs[i] + (offsets[ids[i] + 1] - offsets[ids[i]]);
        }
        if (!gather) {
            // one buffer big enough for the largest bucket sample (at most 256 series)
            int64_t mx = 0;
            for (auto &kv2 : buckets) {
                int64_t t = 0;
                for (int64_t id : kv2.second) t += offsets[id + 1] - offsets[id];
                mx = std::max(mx, t);
            }
            if (cudaMalloc(&gather, (size_t)mx * 4) != cudaSuccess || cudaMalloc(&ko, 256 * 4) != cudaSuccess ||
                cudaMalloc(&no, 256 * 8) != cudaSuccess || cudaMalloc(&dn, 256 * 8) != cudaSuccess ||
                cudaMalloc(&po, 256 * 8) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
                cudaEventCreate(&e1) != cudaSuccess) {
                rc = fail(ctx, MT4G_ENOMEM, "autotune buffers");
                break;
            }
        }
        for (int64_t i = 0; i < n; i++)
            if (cudaMemcpyAsync(gather + offs[i], samples + offsets[ids[i]], (size_t)(offs[i + 1] - offs[i]) * 4,
                                cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
                rc = fail(ctx, MT4G_ECUDA, "autotune gather");
                break;
            }
        if (rc) break;
        float best_ms = 1e30f;
        int32_t best = MT4G_SCAN_SWEEP;
        for (int32_t kpt : {MT4G_SCAN_SWEEP, 1, 2, 4}) {
            ctx->forced_kpt = kpt;
            float ms = 0.f;
            for (int rep = 0; rep < 3 && !rc; rep++) {  // first call warms up, the minimum of the rest counts
                cudaEventRecord(e0, st);
                rc = scan_body(ctx, gather, offs.data(), stp.data(), n, MT4G_MODE_FULL, ko, no, dn, po, st);
                cudaEventRecord(e1, st);
                if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = fail(ctx, MT4G_ECUDA, "autotune timing");
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep == 1 || (rep > 1 && t < ms)) ms = t;
            }
            if (rc) break;
            // the run sweep counts for a bucket only if it takes most of its series (at most 1536
            // distinct values): the others would run as slices inside the sweep kernel, which
            // holds half the warps of the slice kernel, and a whole batch would pay for that
            const bool usable = kpt != MT4G_SCAN_SWEEP || 2 * (int64_t)ctx->h_hdr->unswept <= n;
            if (usable && ms < best_ms) {
                best_ms = ms;
                best = kpt;
            }
        }
        if (rc) break;
        ctx->tune[kv.first] = best;
    }
    ctx->forced_kpt = was_forced;
    ctx->use_graph = was_graph;
    ctx->timing = was_timing;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(gather);
    cudaFree(ko);
    cudaFree(no);
    cudaFree(dn);
    cudaFree(po);
    return rc;
}

extern "C" int mt4g_autotune_save(mt4g_ctx *ctx, const char *path) {
    if (!ctx || !path) return MT4G_EINVAL;
    FILE *f = fopen(path, "w");
    if (!f) return fail(ctx, MT4G_EINVAL, "cannot open %s", path);
    fprintf(f, "# log2(T) log2(m) scan-tile\n");
    for (auto &kv : ctx->tune) fprintf(f, "%d %d %d\n", kv.first.first, kv.first.second, kv.second);
    fclose(f);
    return MT4G_OK;
}

extern "C" int mt4g_autotune_load(mt4g_ctx *ctx, const char *path) {
    if (!ctx || !path) return MT4G_EINVAL;
    FILE *f = fopen(path, "r");
    if (!f) return fail(ctx, MT4G_EINVAL, "cannot open %s", path);
    std::map<std::pair<int, int>, int32_t> t;
    char line[256];
    while (fgets(line, sizeof(line), f)) {
        if (line[0] == '#') continue;
        int a = 0, b = 0, k = 0;
        if (sscanf(line, "%d %d %d", &a, &b, &k) != 3 || (k != 1 && k != 2 && k != 4 && k != MT4G_SCAN_SWEEP)) {
            fclose(f);
            return fail(ctx, MT4G_EINVAL, "%s: bad line", path);
        }
        t[{a, b}] = k;
    }
    fclose(f);
    ctx->tune = t;
    return MT4G_OK;
}

extern "C" int mt4g_autotune_get(mt4g_ctx *ctx, int32_t T, int32_t m) {
    if (!ctx || T < 1 || m < 1) return MT4G_EINVAL;
    return pick_kpt(ctx, T, m);
}
