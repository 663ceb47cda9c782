// Per-series LSD radix sort of the latency samples, carrying step labels, and
// the run table of distinct values.
//
// The ECDFs of Sec. II-C-1 are read off the pooled samples in value order, so each
// series is sorted once: ascending by value, equal values in step order (the input
// is step-major and every pass is stable).  One CTA owns one series and runs all of
// its 8-bit digit passes itself; the number of passes is the smallest even number
// covering the series' largest value, so the result always lands in keyA/labA.
// Passes keep the series' ping-pong buffers hot in L2 (a 64 K-sample series is
// 768 KB across both buffers), so HBM sees roughly one read of the input and one
// write of the sorted labels.
//
// Within a 4096-sample tile, each warp ranks its 256 samples with match.any
// (stable: item-major, then lane order), per-warp digit counts are scanned across
// warps, and a running per-digit base carries the order across tiles.
#include "mt4g_internal.cuh"

namespace mt4g {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

// Exclusive scan of s_in[0..255] into s_out[0..255] by the first 256 threads.
// Must be called by all threads of the block (contains __syncthreads).
__device__ void scan256(const uint32_t *s_in, uint32_t *s_out, uint32_t *s_tmp) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t v = 0, incl = 0;
    if (tid < 256) {
        v = s_in[tid];
        incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_tmp[warp] = incl;
    }
    __syncthreads();
    if (tid < 256) {
        uint32_t wbase = 0;
        for (int w = 0; w < warp; w++) wbase += s_tmp[w];
        s_out[tid] = wbase + incl - v;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kSortThreads, 2)
sort_series_kernel(const uint32_t *__restrict__ samples, SeriesDesc *__restrict__ desc,
                   const int32_t *__restrict__ order, uint32_t *__restrict__ keyA, uint32_t *__restrict__ keyB,
                   uint16_t *__restrict__ labA, uint16_t *__restrict__ labB, int32_t *__restrict__ runs) {
    __shared__ uint32_t s_wc[kSortWarps][256];  // per-warp digit counts, then offsets
    __shared__ uint32_t s_base[256];            // running scatter base of each digit
    __shared__ uint32_t s_hist[256];
    __shared__ uint32_t s_tmp[32];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s = order[blockIdx.x];
    const SeriesDesc d = desc[s];
    const int64_t off = d.off;
    const int32_t m = d.m;
    const int32_t N = d.T * m;

    // ---- largest value -> number of 8-bit passes (even, >= 2)
    uint32_t vmax = 0;
    for (int i = tid; i < N; i += kSortThreads) vmax = max(vmax, __ldg(samples + off + i));
    vmax = __reduce_max_sync(kFull, vmax);
    if (lane == 0) s_tmp[warp] = vmax;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = lane < kSortWarps ? s_tmp[lane] : 0u;
        v = __reduce_max_sync(kFull, v);
        if (lane == 0) s_tmp[31] = v;
    }
    __syncthreads();
    vmax = s_tmp[31];
    __syncthreads();
    const int bits = vmax ? 32 - __clz(vmax) : 0;
    int passes = (bits + 7) / 8;
    passes = max(2, (passes + 1) & ~1);

    for (int p = 0; p < passes; p++) {
        const int shift = 8 * p;
        const uint32_t *src_key = (p == 0) ? samples + off : ((p & 1) ? keyB : keyA) + off;
        const uint16_t *src_lab = ((p & 1) ? labB : labA) + off;
        uint32_t *dst_key = ((p & 1) ? keyA : keyB) + off;
        uint16_t *dst_lab = ((p & 1) ? labA : labB) + off;

        // digit histogram of the whole series
        if (tid < 256) s_hist[tid] = 0;
        __syncthreads();
        for (int b0 = 0; b0 < N; b0 += kSortThreads) {
            const int i = b0 + tid;
            const bool valid = i < N;
            const unsigned vm = __ballot_sync(kFull, valid);
            if (valid) {
                const uint32_t dg = (src_key[i] >> shift) & 255u;
                const unsigned peers = __match_any_sync(vm, dg);
                if ((int)(__ffs(peers) - 1) == lane) atomicAdd(&s_hist[dg], (uint32_t)__popc(peers));
            }
        }
        __syncthreads();
        scan256(s_hist, s_base, s_tmp);

        for (int tb = 0; tb < N; tb += kSortTile) {
            for (int j = lane; j < 256; j += 32) s_wc[warp][j] = 0;
            __syncwarp();
            uint32_t key[kSortItems], rk[kSortItems];
            uint16_t lb[kSortItems];
#pragma unroll
            for (int it = 0; it < kSortItems; it++) {
                const int e = tb + warp * (32 * kSortItems) + it * 32 + lane;
                const bool valid = e < N;
                key[it] = 0;
                lb[it] = 0;
                rk[it] = 0;
                if (valid) {
                    key[it] = src_key[e];
                    lb[it] = (p == 0) ? (uint16_t)(e / m) : src_lab[e];
                }
                const unsigned vm = __ballot_sync(kFull, valid);
                if (valid) {
                    const uint32_t dg = (key[it] >> shift) & 255u;
                    const unsigned peers = __match_any_sync(vm, dg);
                    const int leader = __ffs(peers) - 1;
                    uint32_t old = 0;
                    if (lane == leader) {
                        old = s_wc[warp][dg];
                        s_wc[warp][dg] = old + (uint32_t)__popc(peers);
                    }
                    old = __shfl_sync(peers, old, leader);
                    rk[it] = old + (uint32_t)__popc(peers & lanemask_lt());
                }
                __syncwarp();
            }
            __syncthreads();
            if (tid < 256) {
                uint32_t run = s_base[tid];
#pragma unroll
                for (int w = 0; w < kSortWarps; w++) {
                    const uint32_t c = s_wc[w][tid];
                    s_wc[w][tid] = run;
                    run += c;
                }
                s_base[tid] = run;
            }
            __syncthreads();
#pragma unroll
            for (int it = 0; it < kSortItems; it++) {
                const int e = tb + warp * (32 * kSortItems) + it * 32 + lane;
                if (e < N) {
                    const uint32_t dg = (key[it] >> shift) & 255u;
                    const uint32_t pos = s_wc[warp][dg] + rk[it];
                    dst_key[pos] = key[it];
                    dst_lab[pos] = lb[it];
                }
            }
            __syncthreads();
        }
    }

    // ---- run table: start of every run of equal values, then N
    const uint32_t *fk = keyA + off;
    int32_t *rt = runs + d.run_base;
    uint32_t count = 0;
    for (int tb = 0; tb < N; tb += kSortThreads) {
        const int i = tb + tid;
        const bool flag = i < N && (i == 0 || fk[i] != fk[i - 1]);
        const unsigned b = __ballot_sync(kFull, flag);
        if (lane == 0) s_tmp[warp] = (uint32_t)__popc(b);
        __syncthreads();
        uint32_t before = 0, total = 0;
        for (int w = 0; w < kSortWarps; w++) {
            const uint32_t c = s_tmp[w];
            if (w < warp) before += c;
            total += c;
        }
        if (flag) rt[count + before + (uint32_t)__popc(b & lanemask_lt())] = i;
        count += total;
        __syncthreads();
    }
    if (tid == 0) {
        rt[count] = N;
        desc[s].nruns = (int32_t)count;
    }
}

// ---- Eq. 2 reduction (paper Sec. IV-B-1): S_t = sqrt(sum_j (r_tj - min r)^2), then
// each S_t replaced by its rank among the series' values (count of strictly smaller
// values).  Ranks preserve order and ties exactly, so the KS test on the ranks is
// the KS test on S.  The sum runs in j order with explicit round-to-nearest
// operations (no contraction into FMA).
__global__ void __launch_bounds__(256)
reduce_rank_kernel(const uint32_t *__restrict__ samples, const SeriesDesc *__restrict__ desc, double *red,
                   uint32_t *rank_out) {
    __shared__ uint32_t s_min[32];
    __shared__ double s_tile[1024];
    const int s = blockIdx.x;
    const SeriesDesc d = desc[s];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t N = (int64_t)d.T * d.m;
    const uint32_t *x = samples + d.off;
    uint32_t mn = 0xffffffffu;
    for (int64_t i = tid; i < N; i += blockDim.x) mn = min(mn, __ldg(x + i));
    mn = __reduce_min_sync(kFull, mn);
    if (lane == 0) s_min[warp] = mn;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = lane < (int)(blockDim.x / 32) ? s_min[lane] : 0xffffffffu;
        v = __reduce_min_sync(kFull, v);
        if (lane == 0) s_min[31] = v;
    }
    __syncthreads();
    mn = s_min[31];
    double *r = red + d.step_base;
    for (int t = tid; t < d.T; t += blockDim.x) {
        double acc = 0.0;
        const uint32_t *row = x + (int64_t)t * d.m;
        for (int j = 0; j < d.m; j++) {
            const double v = (double)(__ldg(row + j) - mn);
            acc = __dadd_rn(acc, __dmul_rn(v, v));
        }
        r[t] = __dsqrt_rn(acc);
    }
    __syncthreads();
    // ranks: number of strictly smaller reduced values
    for (int t0 = 0; t0 < d.T; t0 += blockDim.x) {
        const int t = t0 + tid;
        const double v = t < d.T ? r[t] : 0.0;
        uint32_t rank = 0;
        for (int u0 = 0; u0 < d.T; u0 += 1024) {
            __syncthreads();
            for (int u = tid; u < 1024; u += blockDim.x) s_tile[u] = (u0 + u < d.T) ? r[u0 + u] : 0.0;
            __syncthreads();
            const int nu = min(1024, d.T - u0);
            for (int u = 0; u < nu; u++) rank += s_tile[u] < v;
        }
        if (t < d.T) rank_out[d.step_base + t] = rank;
    }
}

}  // namespace

cudaError_t launch_sort(const uint32_t *samples, SeriesDesc *desc, const int32_t *order, int64_t S,
                        uint32_t *keyA, uint32_t *keyB, uint16_t *labA, uint16_t *labB, int32_t *runs,
                        cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    sort_series_kernel<<<(unsigned)S, kSortThreads, 0, st>>>(samples, desc, order, keyA, keyB, labA, labB, runs);
    return cudaGetLastError();
}

cudaError_t launch_reduce_rank(const uint32_t *samples, const SeriesDesc *raw_desc, int64_t S, double *red,
                               uint32_t *rank_out, cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    reduce_rank_kernel<<<(unsigned)S, 256, 0, st>>>(samples, raw_desc, red, rank_out);
    return cudaGetLastError();
}

}  // namespace mt4g
