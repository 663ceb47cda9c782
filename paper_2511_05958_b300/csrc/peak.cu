// mt4g_int32_peak: the measured integer issue rate that bounds the exact scan.
//
// The scan's inner step, for one split k and one distinct value x, is f = H c_L - a C,
// |f| and a running maximum: two multiply-adds, an absolute value and a max on 32-bit
// integers.  This kernel runs that same mix on every SM with enough independent chains
// per thread to hide the pipeline latency, so its rate is the ceiling the scan's
// (split, distinct value) evaluations can approach on this GPU at its current clocks.
// It touches no memory except one conditional store that keeps the chains alive.
#include "mt4g_internal.cuh"

// External linkage: the conditional store to it is observable, so the chains stay live.
__device__ uint32_t mt4g_peak_sink;

namespace {

constexpr int kChains = 8;
constexpr int kOpsPerStep = 4;  // IMAD, IMAD, IABS, IMNMX per chain and iteration

__global__ void __launch_bounds__(256) int32_peak_kernel(uint32_t H, uint32_t a0, uint32_t C0, int iters) {
    uint32_t cl[kChains], mx[kChains];
    const uint32_t a = a0 + (threadIdx.x & 7);
#pragma unroll
    for (int c = 0; c < kChains; c++) {
        cl[c] = threadIdx.x + 3u * c;
        mx[c] = 0;
    }
    uint32_t C = C0 + blockIdx.x;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) {
            const int32_t f = (int32_t)(H * cl[c] - a * (C + c));
            const uint32_t af = (uint32_t)(f < 0 ? -f : f);
            mx[c] = max(mx[c], af);
            cl[c] = mx[c];  // the next step's count depends on this one: no folding
        }
    }
    uint32_t r = 0;
#pragma unroll
    for (int c = 0; c < kChains; c++) r ^= mx[c];
    if (r == 0x1e3779b9u) mt4g_peak_sink = r;  // below 2^31, the range of |f|
}

}  // namespace

extern "C" int mt4g_int32_peak(int device, double *tops_out) {
    if (!tops_out) return MT4G_EINVAL;
    *tops_out = 0.0;
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || device < 0 || device >= dev_count) return MT4G_ECUDA;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return MT4G_ECUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int threads = 256, blocks = sms * 8, iters = 1 << 14;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = MT4G_OK;
    float best = 0.f;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        rc = MT4G_ECUDA;
    } else {
        for (int rep = 0; rep < 5 && rc == MT4G_OK; rep++) {
            cudaEventRecord(e0, st);
            int32_peak_kernel<<<blocks, threads, 0, st>>>(512u, 1u, 65536u, iters);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
                rc = MT4G_ECUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep >= 2 && (best == 0.f || ms < best)) best = ms;  // first two are warm-up
        }
    }
    if (rc == MT4G_OK && best > 0.f) {
        const double ops = (double)blocks * threads * iters * kChains * kOpsPerStep;
        *tops_out = ops / (best * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaSetDevice(prev);
    return rc;
}
