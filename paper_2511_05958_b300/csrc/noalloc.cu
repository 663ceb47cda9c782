// mt4g_ks_scan_noalloc: the top-level scan of a small batch without any allocation.
//
// Some callers cannot allocate device memory at all: code that runs inside a memory pool
// or arena owned by someone else (a framework's caching allocator, an embedded runtime
// with a fixed budget), or processes whose allocation calls are forbidden after start-up.
// For them this entry point runs the same sort and all-splits scan as mt4g_ks_scan, but
// every scratch buffer is carved from one file-scope device array of kNoAllocBytes, which
// each GPU that loads the library holds until the process exits.  Host-side tables go
// through a static host buffer, so the call allocates no host memory either.
//
// Limits (checked before any GPU work, MT4G_EINVAL beyond them): at most kNoAllocSeries
// series, kNoAllocSamples samples and kNoAllocSteps steps in total.
//
// The array is shared by every call on a device and keeps the last call's contents; the
// parts that must start at zero (queue flags and counters) are cleared by each call.
// Calls whose GPU work overlaps (on different streams, or from several host threads)
// race on the array; host-side staging is serialised by a mutex.  The first call on a
// device looks up the array's device address (cudaGetSymbolAddress) and caches it.  The
// call returns after its results are written (it synchronises the stream) so that it can
// report device-side status without a context; when an enqueue fails part way, it still
// waits for the work already enqueued, so that nothing of a failed call runs on the array
// after it returns.
#include <cstring>
#include <mutex>

#include "mt4g_internal.cuh"

using namespace mt4g;

namespace {

constexpr int64_t kNoAllocSeries = 4096;
constexpr int64_t kNoAllocSamples = 1 << 19;
constexpr int64_t kNoAllocSteps = 1 << 16;
constexpr size_t kNoAllocBytes = 12u << 20;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_mutex;

// host staging: header, descriptors, sort order, queue order, slice bases
alignas(64) unsigned char g_host_stage[sizeof(QueueHeader) + kNoAllocSeries * (sizeof(SeriesDesc) + 16) + 256];

struct Layout {
    size_t off_hdr, off_desc, off_order, off_qorder, off_base, off_keyA, off_keyB, off_labA, off_labB, off_runs,
        off_items, off_ready, off_gcount, end;
};

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

Layout layout(int64_t S, int64_t Ntot, unsigned long long cap) {
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = up256(o + bytes);
        return at;
    };
    L.off_hdr = take(sizeof(QueueHeader));
    L.off_desc = take(S * sizeof(SeriesDesc));
    L.off_order = take(S * sizeof(int32_t));
    L.off_qorder = take(S * sizeof(int32_t));
    L.off_base = take(S * sizeof(int64_t));
    L.off_keyA = take(Ntot * sizeof(uint32_t));
    L.off_keyB = take(Ntot * sizeof(uint32_t));
    L.off_labA = take(Ntot * sizeof(uint16_t));
    L.off_labB = take(Ntot * sizeof(uint16_t));
    L.off_runs = take((Ntot + S) * sizeof(int32_t));
    L.off_items = take(cap * sizeof(WorkItem));
    L.off_ready = take(cap * sizeof(int32_t));
    L.off_gcount = take(cap * sizeof(uint32_t));
    L.end = o;
    return L;
}

// The worst case of the stated limits must fit the array.
static_assert(sizeof(QueueHeader) + kNoAllocSeries * (sizeof(SeriesDesc) + 16) +
                      kNoAllocSamples * (4 + 4 + 2 + 2 + 4) + (kNoAllocSeries + 1) * 4 +
                      (kNoAllocSteps / 32 + kNoAllocSeries + 64) * (sizeof(WorkItem) + 8) + 16 * 256 <=
                  kNoAllocBytes,
              "no-allocation scratch array too small for its limits");

int scratch_for_device(int dev, void **ptr) {
    if (dev < 0 || dev >= kMaxDevices) return MT4G_ECUDA;
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MT4G_ECUDA;
        g_scratch_ptr[dev] = p;
    }
    *ptr = g_scratch_ptr[dev];
    return MT4G_OK;
}

}  // namespace

extern "C" int mt4g_ks_scan_noalloc(const uint32_t *samples, const int64_t *offsets, const int32_t *steps, int64_t S,
                                    int32_t *k_out, int64_t *dnum_out, int64_t *dden_out, double *p_out,
                                    void *cuda_stream) {
    if (S < 0 || S > kNoAllocSeries) return MT4G_EINVAL;
    if (S == 0) return MT4G_OK;
    if (!samples || !offsets || !steps || !k_out || !dnum_out || !dden_out || !p_out) return MT4G_EINVAL;
    if (offsets[0] != 0) return MT4G_EINVAL;
    int64_t ntot = 0, sumT = 0, n_init = 0;
    for (int64_t s = 0; s < S; s++) {
        const int64_t n = offsets[s + 1] - offsets[s];
        const int32_t T = steps[s];
        if (T < 2 || T > MT4G_MAX_STEPS || n <= 0 || n % T != 0) return MT4G_EINVAL;
        ntot += n;
        sumT += T;
        n_init += seg_chunks(T, 1, 1);
    }
    if (ntot > kNoAllocSamples || sumT > kNoAllocSteps) return MT4G_EINVAL;
    const unsigned long long cap = (unsigned long long)n_init + 64;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MT4G_ECUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    void *base = nullptr;
    if (scratch_for_device(dev, &base)) return MT4G_ECUDA;
    const Layout L = layout(S, ntot, cap);
    if (L.end > kNoAllocBytes) return MT4G_EINVAL;
    char *db = (char *)base;
    cudaStream_t st = (cudaStream_t)cuda_stream;

    // host tables in the static staging buffer: header, descriptors, orders, slice bases
    unsigned char *h = g_host_stage;
    QueueHeader hq{};
    hq.tail = (unsigned long long)n_init;
    hq.pending = (long long)n_init;
    hq.cap = cap;
    memcpy(h, &hq, sizeof(hq));
    SeriesDesc *hd = (SeriesDesc *)(h + sizeof(QueueHeader));
    int32_t *horder = (int32_t *)(hd + S);
    int64_t *hbase = (int64_t *)(horder + S + (S & 1));
    int64_t sb = 0, nb = 0;
    for (int64_t s = 0; s < S; s++) {
        SeriesDesc d{};
        d.off = offsets[s];
        d.T = steps[s];
        d.m = (int32_t)((offsets[s + 1] - offsets[s]) / steps[s]);
        d.step_base = sb;
        d.run_base = d.off + s;
        d.kpt = 1;
        hd[s] = d;
        horder[s] = (int32_t)s;
        hbase[s] = nb;
        sb += d.T;
        nb += seg_chunks(d.T, 1, 1);
    }
    // After the first enqueue, a failure drains the stream before returning: the next call
    // must not find this call's copies or kernels still working on the shared array.
#define NA_TRY(expr)                            \
    do {                                        \
        if ((expr) != cudaSuccess) {            \
            (void)cudaStreamSynchronize(st);    \
            (void)cudaGetLastError();           \
            return MT4G_ECUDA;                  \
        }                                       \
    } while (0)
    NA_TRY(cudaMemcpyAsync(db + L.off_hdr, h, sizeof(QueueHeader), cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(db + L.off_desc, hd, S * sizeof(SeriesDesc), cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(db + L.off_order, horder, S * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(db + L.off_qorder, horder, S * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(db + L.off_base, hbase, S * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    // what must start at zero: the queue's ready flags and group counters
    NA_TRY(cudaMemsetAsync(db + L.off_ready, 0, cap * sizeof(int32_t), st));
    NA_TRY(cudaMemsetAsync(db + L.off_gcount, 0, cap * sizeof(uint32_t), st));

    QueueHeader *q = (QueueHeader *)(db + L.off_hdr);
    SeriesDesc *desc = (SeriesDesc *)(db + L.off_desc);
    WorkItem *items = (WorkItem *)(db + L.off_items);
    int32_t *ready = (int32_t *)(db + L.off_ready);
    uint32_t *gcount = (uint32_t *)(db + L.off_gcount);
    const uint32_t epoch = 1u << 16;
    NA_TRY(launch_init_items(desc, (const int32_t *)(db + L.off_qorder), (const int64_t *)(db + L.off_base), S, 1,
                             1, items, ready, gcount, epoch, st));
    NA_TRY(launch_sort(samples, desc, (const int32_t *)(db + L.off_order), S, (uint32_t *)(db + L.off_keyA),
                       (uint32_t *)(db + L.off_keyB), (uint16_t *)(db + L.off_labA), (uint16_t *)(db + L.off_labB),
                       (int32_t *)(db + L.off_runs), nullptr, st));
    RunParams R{};
    R.desc = desc;
    R.lab = (const uint16_t *)(db + L.off_labA);
    R.runs = (const int32_t *)(db + L.off_runs);
    R.q = q;
    R.items = items;
    R.ready = ready;
    R.gcount = gcount;
    R.mode = kRunScan;
    R.min_seg = 1;
    R.wait_limit_ns = 5000000000LL;
    R.k_out = k_out;
    R.dnum_out = dnum_out;
    R.dden_out = dden_out;
    R.p_out = p_out;
    const int grid = queue_grid(dev);
    NA_TRY(grid > 0 ? cudaSuccess : cudaErrorInvalidConfiguration);
    NA_TRY(launch_queue_run(R, grid, epoch, st));
    int32_t status = 0;
    NA_TRY(cudaMemcpyAsync(&status, &q->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    NA_TRY(cudaStreamSynchronize(st));
#undef NA_TRY
    if (status & kStatusTimeout) return MT4G_ETIMEOUT;
    if (status & kStatusQueueFull) return MT4G_ECAPACITY;
    return MT4G_OK;
}
