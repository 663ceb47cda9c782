// C ABI of libmt4g: context, argument validation, workspace, and the call sequence
//   (reduce+rank for Eq. 2 mode) -> per-series radix sort + run table ->
//   persistent work-queue kernel (scan, p-value, segmentation) -> collect.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "mt4g_internal.cuh"

using namespace mt4g;

struct mt4g_ctx {
    int device = 0;
    int grid = 0;
    std::string err;
    long long wait_limit_ns = 5000000000LL;

    void *ws = nullptr;  // device workspace
    size_t ws_bytes = 0;
    void *pin = nullptr;  // pinned host staging for per-call tables
    size_t pin_bytes = 0;
    cudaEvent_t pin_free = nullptr;  // recorded after the last upload out of `pin`
    QueueHeader *h_hdr = nullptr;     // pinned: queue header (status, work) of the last call
    cudaStream_t last_stream = nullptr;
    bool have_last = false;      // some call has enqueued work on last_stream
    bool last_enqueued = false;  // the most recent call enqueued work (its status is in h_hdr)

    int32_t forced_kpt = 0;  // 0: per-series choice; 1, 2, 4: every series

    // stage timing: events of the last kTimingRing calls
    static constexpr int kTimingRing = 64;
    static constexpr int kMarks = 5;
    bool timing = false;
    bool events_made = false;
    cudaEvent_t ev[kTimingRing][kMarks] = {};
    int ring_pos = 0;
    int ring_count = 0;

    // work-queue ready flags carry an epoch so they need no clearing between calls
    uint32_t call_counter = 0;
    size_t ready_off = (size_t)-1;
    unsigned long long ready_cap = 0;
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
    int64_t n_init = 0;                // top-level slices
    unsigned long long cap = 0;
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
    WorkItem *items;
    int32_t *ready;
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
    B.red = c.take<double>(P.reduced ? P.sumT : 0);
    B.rank = c.take<uint32_t>(P.reduced ? P.sumT : 0);
    B.items = c.take<WorkItem>(P.cap);
    B.ready = c.take<int32_t>(P.cap);
    *ready_off = (size_t)((char *)B.ready - (char *)base);
    return c.off + 256;
}

// Record stage boundary `i` of the current call when stage timing is on.
void mark(mt4g_ctx *ctx, int i, cudaStream_t st) {
    if (ctx->timing) cudaEventRecord(ctx->ev[ctx->ring_pos][i], st);
}

// Scan tile for a series: split groups of 32 per warp work item.  A forced value
// (MT4G_OPT_SCAN_KPT) wins; otherwise the autotuned table, else a size heuristic.
int32_t pick_kpt(const mt4g_ctx *ctx, int32_t T, int32_t m) {
    if (ctx->forced_kpt) return ctx->forced_kpt;
    (void)T;
    (void)m;
    return 1;
}

// Validate the host tables and build the per-call plan.
int make_plan(mt4g_ctx *ctx, const int64_t *offsets, const int32_t *steps, int64_t S, int32_t mode,
              int32_t min_seg, Plan &P) {
    if (S < 0) return fail(ctx, MT4G_EINVAL, "S must be >= 0 (got %lld)", (long long)S);
    if (S > 0 && (!offsets || !steps)) return fail(ctx, MT4G_EINVAL, "offsets and steps must be non-NULL");
    if (S > (int64_t)INT32_MAX) return fail(ctx, MT4G_EINVAL, "too many series");
    if (mode != MT4G_MODE_FULL && mode != MT4G_MODE_REDUCED)
        return fail(ctx, MT4G_EINVAL, "mode must be MT4G_MODE_FULL or MT4G_MODE_REDUCED (got %d)", mode);
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
        d.kpt = pick_kpt(ctx, d.T, d.m);
        P.desc[s] = d;
        sumT += T;
        ntot += (int64_t)d.T * d.m;
    }
    P.sumT = sumT;
    P.Ntot = ntot;
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
    P.item_base.resize(S);
    int64_t nb = 0;
    for (int64_t i = 0; i < S; i++) {
        P.item_base[i] = nb;
        nb += seg_chunks(P.desc[P.qorder[i]].T, min_seg, P.desc[P.qorder[i]].kpt);
    }
    P.n_init = nb;
    // slices of the children of accepted splits: a split of a segment adds at most
    // two slices beyond the parent's, so 2 per step plus the top level bounds them
    // for the usual few change points per series; overflow is reported.
    P.cap = (unsigned long long)nb + 4ull * (unsigned long long)sumT + 1024ull;
    return MT4G_OK;
}

int ensure_workspace(mt4g_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->ws_bytes) return MT4G_OK;
    if (ctx->have_last) CUDA_TRY(ctx, cudaStreamSynchronize(ctx->last_stream));
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

// Everything a call enqueues up to (and including) the work-queue kernel.
int enqueue_pipeline(mt4g_ctx *ctx, const uint32_t *samples, Plan &P, RunParams &R, Buffers &B, cudaStream_t st) {
    size_t ready_off = 0;
    const size_t need = carve(nullptr, P, B, &ready_off);
    int rc = ensure_workspace(ctx, need);
    if (rc) return rc;
    carve(ctx->ws, P, B, &ready_off);

    // epoch of this call's ready flags; clear them when the layout changed or the epoch wraps
    ctx->call_counter++;
    uint32_t e = ctx->call_counter & 0x7fff;
    const bool fresh = ready_off != ctx->ready_off || P.cap > ctx->ready_cap || e == 0;
    if (e == 0) {
        ctx->call_counter++;
        e = ctx->call_counter & 0x7fff;
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
    rc = ensure_pinned(ctx, bytes_hdr + bytes_desc + bytes_raw + bytes_order + bytes_items + bytes_ready + 64);
    if (rc) return rc;
    char *h = (char *)ctx->pin;
    QueueHeader hq{};
    hq.head = 0;
    hq.tail = n_items;
    hq.pending = (long long)n_items;
    hq.status = 0;
    hq.cap = P.cap;
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

    CUDA_TRY(ctx, cudaMemcpyAsync(B.q, h, bytes_hdr, cudaMemcpyHostToDevice, st));
    if (bytes_desc) CUDA_TRY(ctx, cudaMemcpyAsync(B.desc, h + o_desc, bytes_desc, cudaMemcpyHostToDevice, st));
    if (bytes_raw) CUDA_TRY(ctx, cudaMemcpyAsync(B.raw_desc, h + o_raw, bytes_raw, cudaMemcpyHostToDevice, st));
    if (bytes_order) CUDA_TRY(ctx, cudaMemcpyAsync(B.order, h + o_order, bytes_order, cudaMemcpyHostToDevice, st));
    if (bytes_items) CUDA_TRY(ctx, cudaMemcpyAsync(B.qorder, h + o_items, bytes_items, cudaMemcpyHostToDevice, st));
    if (bytes_ready)
        CUDA_TRY(ctx, cudaMemcpyAsync(B.item_base, h + o_ready, bytes_ready, cudaMemcpyHostToDevice, st));
    CUDA_TRY(ctx, cudaEventRecord(ctx->pin_free, st));
    CUDA_TRY(ctx, launch_init_items(B.desc, B.qorder, B.item_base, P.S, P.min_seg, B.items, B.ready, epoch, st));
    mark(ctx, 1, st);

    const uint32_t *sort_in = samples;
    if (P.reduced) {
        CUDA_TRY(ctx, launch_reduce_rank(samples, B.raw_desc, P.S, B.red, B.rank, st));
        sort_in = B.rank;
    }
    CUDA_TRY(ctx, launch_sort(sort_in, B.desc, B.order, P.S, B.keyA, B.keyB, B.labA, B.labB, B.runs, st));
    mark(ctx, 2, st);

    R = RunParams{};
    R.desc = B.desc;
    R.lab = B.labA;
    R.runs = B.runs;
    R.q = B.q;
    R.items = B.items;
    R.ready = B.ready;
    R.min_seg = P.min_seg;
    R.wait_limit_ns = ctx->wait_limit_ns;
    R.cp_flag = B.cp_flag;
    R.cp_num = B.cp_num;
    R.cp_den = B.cp_den;
    R.cp_p = B.cp_p;
    return (int)epoch;  // >= 0
}

int finish_call(mt4g_ctx *ctx, Buffers &B, cudaStream_t st) {
    mark(ctx, 4, st);
    if (ctx->timing) {
        ctx->ring_pos = (ctx->ring_pos + 1) % mt4g_ctx::kTimingRing;
        ctx->ring_count = std::min(ctx->ring_count + 1, mt4g_ctx::kTimingRing);
    }
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_hdr, B.q, sizeof(QueueHeader), cudaMemcpyDeviceToHost, st));
    ctx->last_stream = st;
    ctx->have_last = true;
    ctx->last_enqueued = true;
    return MT4G_OK;
}

int begin_call(mt4g_ctx *ctx) {
    if (!ctx) return MT4G_EINVAL;
    ctx->err.clear();
    ctx->last_enqueued = false;
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
    if (c->grid <= 0) {
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
        if (value != 0 && value != 1 && value != 2 && value != 4)
            return fail(c, MT4G_EINVAL, "scan tile must be 0 (automatic), 1, 2 or 4");
        c->forced_kpt = (int32_t)value;
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
    const int32_t st = c->h_hdr->status;
    if (st & kStatusTimeout) return fail(c, MT4G_ETIMEOUT, "a bounded device-side wait expired");
    if (st & kStatusQueueFull) return fail(c, MT4G_ECAPACITY, "work queue capacity exceeded");
    if (st & kStatusCapacity) return fail(c, MT4G_ECAPACITY, "a series has more than max_cp change points");
    return MT4G_OK;
}

int mt4g_ks_scan(mt4g_ctx *ctx, const uint32_t *samples, const int64_t *offsets, const int32_t *steps, int64_t S,
                 int32_t mode, int32_t *k_out, int64_t *dnum_out, int64_t *dden_out, double *p_out,
                 void *cuda_stream) {
    int rc = begin_call(ctx);
    if (rc) return rc;
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
    CUDA_TRY(ctx, launch_queue_run(R, ctx->grid, (uint32_t)epoch, st));
    mark(ctx, 3, st);
    return finish_call(ctx, B, st);
}

int mt4g_ks_segment(mt4g_ctx *ctx, const uint32_t *samples, const int64_t *offsets, const int32_t *steps, int64_t S,
                    double alpha, int32_t min_seg, int32_t max_cp, int32_t mode, int32_t *cp_count, int32_t *cp_idx,
                    int64_t *dnum, int64_t *dden, double *p, void *cuda_stream) {
    int rc = begin_call(ctx);
    if (rc) return rc;
    if (!(alpha > 0.0 && alpha < 1.0)) return fail(ctx, MT4G_EINVAL, "alpha must be in (0, 1)");
    if (max_cp < 0) return fail(ctx, MT4G_EINVAL, "max_cp must be >= 0");
    if (S > 0 && (!samples || !cp_count || (max_cp > 0 && (!cp_idx || !dnum || !dden || !p))))
        return fail(ctx, MT4G_EINVAL, "NULL device pointer");
    Plan P;
    rc = make_plan(ctx, offsets, steps, S, mode, min_seg, P);
    if (rc) return rc;
    if (S == 0) return MT4G_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    Buffers B;
    RunParams R;
    mark(ctx, 0, st);
    const int epoch = enqueue_pipeline(ctx, samples, P, R, B, st);
    if (epoch < 0) return epoch;
    R.mode = kRunSegment;
    R.alpha = alpha;
    CUDA_TRY(ctx, cudaMemsetAsync(B.cp_flag, 0, (size_t)P.sumT, st));
    CUDA_TRY(ctx, launch_queue_run(R, ctx->grid, (uint32_t)epoch, st));
    mark(ctx, 3, st);
    CUDA_TRY(ctx, launch_collect(B.desc, P.S, B.cp_flag, B.cp_num, B.cp_den, B.cp_p, max_cp, cp_count, cp_idx, dnum,
                                 dden, p, B.q, st));
    return finish_call(ctx, B, st);
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
