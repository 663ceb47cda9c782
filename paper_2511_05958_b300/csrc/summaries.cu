// Per-step summaries that the learned change-point proposal reads.
//
// The paper evaluates every index of a series (Sec. IV-B-1 (4)) and notes that change
// points can be shortlisted first to save computation; the shortlisting network reads,
// for each array-size step t, 17 features:
//   i < 16: log2(q_i) - log2(med), q_i the sorted step sample at rank
//           min(m - 1, floor((i + 0.5) m / 16)), med the series' sorted sample at N / 2;
//   16:     log2(1024 + 32 t) - 10, the array size of the step (fetch-granularity
//           steps from 1 KiB, Sec. IV-B-1 (2)), shifted to start at 0.
// Values are read as at least 1.  Features are computed in FP32 and stored as BF16
// (round to nearest even) in rows of kFeatC channels (the last is zero).
//
// Steps of m = 32, 64 or 128 samples: one thread per step.  A warp copies 32 consecutive
// steps into a padded shared-memory stage (cp.async), each thread reads its step's row into
// registers, the warp starts copying its next 32 steps, and each thread sorts its row with
// Batcher's odd-even merge network on compile-time register indices (no shuffles; the
// compiler drops the exchanges that no selected rank depends on).  Other m <= 256: one warp
// per step, a bitonic network with V values per lane and partners across lanes by shuffle,
// then lanes 0..15 pick their quantile; each warp loads its next step while sorting.
#include <cuda_bf16.h>

#include "mt4g_internal.cuh"

namespace mt4g {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSumWarps = 4;  // warps per block (one block per series)
constexpr int kRowMax = 128;  // largest m sorted one step per thread
// stage of one warp: 32 rows of m words at a stride of m + 4 words (16-byte aligned rows; the
// eight lanes of a quarter warp start their 16-byte reads in eight different bank groups)
constexpr int kStageWords = 32 * (kRowMax + 4);
constexpr size_t kSumSmem = (size_t)kSumWarps * kStageWords * sizeof(uint32_t);

__device__ __forceinline__ void cmpx(uint32_t &a, uint32_t &b) {
    const uint32_t lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}

// Batcher's odd-even merge of x[LO, LO + LEN), whose halves are sorted, comparing elements R
// apart: merge the even and the odd subsequences (stride 2R), then exchange neighbours.
template <int LO, int LEN, int R, int N>
__device__ __forceinline__ void oe_merge(uint32_t (&x)[N]) {
    if constexpr (2 * R < LEN) {
        oe_merge<LO, LEN, 2 * R>(x);
        oe_merge<LO + R, LEN, 2 * R>(x);
#pragma unroll
        for (int i = LO + R; i + R < LO + LEN; i += 2 * R) cmpx(x[i], x[i + R]);
    } else {
        cmpx(x[LO], x[LO + R]);
    }
}

template <int LO, int LEN, int N>
__device__ __forceinline__ void oe_sort(uint32_t (&x)[N]) {
    if constexpr (LEN > 1) {
        oe_sort<LO, LEN / 2>(x);
        oe_sort<LO + LEN / 2, LEN / 2>(x);
        oe_merge<LO, LEN, 1>(x);
    }
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ uint32_t bf16_pair(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// Features of the steps of one series with m == N, one thread per step: groups of 32 steps
// warp, warp + kSumWarps, ...; the next group is copied into the stage while this one sorts.
template <int N>
__device__ void summarise_rows(const uint32_t *__restrict__ x0, int T, float lmed, int warp, uint32_t *stage,
                               __nv_bfloat16 *__restrict__ base) {
    static_assert(N % 4 == 0 && N <= kRowMax, "row size");
    constexpr int RS = N + 4;  // row stride in words
    const int lane = threadIdx.x & 31;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(stage);
    const bool vec = (reinterpret_cast<uintptr_t>(x0) & 15) == 0;  // rows of N words stay aligned
    auto issue = [&](int g) {
        const int t0 = g * 32, rows = min(32, T - t0);
        const uint32_t *src = x0 + (int64_t)t0 * N;
        if (vec) {
            constexpr int Q = N / 4;
            for (int p = lane; p < rows * Q; p += 32)
                cp_async16(sbase + (uint32_t)((p / Q) * RS + (p % Q) * 4) * 4u, src + (int64_t)p * 4);
        } else {
            for (int p = lane; p < rows * N; p += 32)
                cp_async4(sbase + (uint32_t)((p / N) * RS + p % N) * 4u, src + p);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if (warp * 32 < T) issue(warp);
    for (int g = warp; g * 32 < T; g += kSumWarps) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncwarp();
        uint32_t x[N];
        const uint4 *row = reinterpret_cast<const uint4 *>(stage + lane * RS);
#pragma unroll
        for (int q = 0; q < N / 4; q++) {
            const uint4 v = row[q];
            x[4 * q] = v.x;
            x[4 * q + 1] = v.y;
            x[4 * q + 2] = v.z;
            x[4 * q + 3] = v.w;
        }
        __syncwarp();
        if ((g + kSumWarps) * 32 < T) issue(g + kSumWarps);
        oe_sort<0, N>(x);
        const int t = g * 32 + lane;
        if (t < T) {
            float f[kFeatC];
#pragma unroll
            for (int i = 0; i < 16; i++) {
                const int rank = ((2 * i + 1) * N) / 32 < N - 1 ? ((2 * i + 1) * N) / 32 : N - 1;
                f[i] = log2f((float)max(x[rank], 1u)) - lmed;
            }
            f[16] = log2f(1024.f + 32.f * (float)t) - 10.f;
            f[17] = 0.f;
            uint32_t *dst = reinterpret_cast<uint32_t *>(base + (int64_t)(2 + t) * kFeatC);
#pragma unroll
            for (int j = 0; j < kFeatC / 2; j++) dst[j] = bf16_pair(f[2 * j], f[2 * j + 1]);
        }
    }
}

// Ascending bitonic sort of 32 V values; lane l holds elements l V .. l V + V - 1.  The
// direction of a compare-exchange depends on the element's index only through bits >= log2 V
// in the stages that cross lanes and in every stage with k > V, so it is computed once per
// lane and stage there; each exchange is then one min or max (selected by a predicate).
template <int V>
__device__ __forceinline__ void bitonic_sort_warp(uint32_t (&x)[V]) {
    const int lane = threadIdx.x & 31;
    const int base = lane * V;
    constexpr int N = 32 * V;
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j < V) {
#pragma unroll
                for (int r = 0; r < V; r++) {
                    const int p = r ^ j;
                    if (p > r) {
                        const bool up = k < V ? ((r & k) == 0) : ((base & k) == 0);
                        const uint32_t lo = min(x[r], x[p]), hi = max(x[r], x[p]);
                        x[r] = up ? lo : hi;
                        x[p] = up ? hi : lo;
                    }
                }
            } else {
                const int lj = j / V;
                const bool takemin = ((base & k) == 0) == ((base & j) == 0);
#pragma unroll
                for (int r = 0; r < V; r++) {
                    const uint32_t o = __shfl_xor_sync(kFull, x[r], lj);
                    x[r] = takemin ? min(x[r], o) : max(x[r], o);
                }
            }
        }
    }
}

// Features of steps warp, warp + kSumWarps, ... of one series; each step's samples are
// loaded one step ahead, so the loads of the next step are in flight while this one is sorted.
template <int V>
__device__ void summarise_steps(const uint32_t *__restrict__ x0, int T, int m, float lmed, int warp,
                                __nv_bfloat16 *__restrict__ base) {
    const int lane = threadIdx.x & 31;
    uint32_t nx[V];
    auto load = [&](int t, uint32_t(&v)[V]) {
        const uint32_t *row = x0 + (int64_t)t * m;
#pragma unroll
        for (int r = 0; r < V; r++) {
            const int e = lane * V + r;
            v[r] = e < m ? __ldg(row + e) : 0xffffffffu;
        }
    };
    if (warp < T) load(warp, nx);
    const int i = lane & 15;
    const int rank = min(m - 1, ((2 * i + 1) * m) / 32);
    for (int t = warp; t < T; t += kSumWarps) {
        uint32_t x[V];
#pragma unroll
        for (int r = 0; r < V; r++) x[r] = nx[r];
        if (t + kSumWarps < T) load(t + kSumWarps, nx);
        bitonic_sort_warp<V>(x);
        uint32_t q = 0;
#pragma unroll
        for (int r = 0; r < V; r++) {
            const uint32_t v = __shfl_sync(kFull, x[r], rank / V);
            if (rank % V == r) q = v;
        }
        float f = 0.f;
        if (lane < 16)
            f = log2f((float)max(q, 1u)) - lmed;
        else if (lane == 16)
            f = log2f(1024.f + 32.f * (float)t) - 10.f;
        if (lane < kFeatC) base[(int64_t)(2 + t) * kFeatC + lane] = __float2bfloat16_rn(f);
    }
}

__global__ void __launch_bounds__(kSumWarps * 32, 3) summaries_kernel(const uint32_t *__restrict__ samples,
                                                        const SeriesDesc *__restrict__ desc,
                                                        __nv_bfloat16 *__restrict__ feat,
                                                        const unsigned long long *__restrict__ gate) {
    if (gate && *gate == 0ull) return;
    const int64_t s = blockIdx.x;
    const SeriesDesc d = desc[s];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float lmed = log2f((float)max(d.median, 1u));
    __nv_bfloat16 *base = feat + row_base(d, s) * kFeatC;
    // zero the two pad rows on each side
    if (warp == 0) {
        for (int c = lane; c < 2 * kFeatC; c += 32) {
            base[c] = __float2bfloat16_rn(0.f);
            base[(int64_t)(d.T + 2) * kFeatC + c] = __float2bfloat16_rn(0.f);
        }
    }
    const uint32_t *x0 = samples + d.off;
    extern __shared__ __align__(16) uint32_t sum_stage[];
    uint32_t *stage = sum_stage + warp * kStageWords;
    if (d.m == 128)
        summarise_rows<128>(x0, d.T, lmed, warp, stage, base);
    else if (d.m == 64)
        summarise_rows<64>(x0, d.T, lmed, warp, stage, base);
    else if (d.m == 32)
        summarise_rows<32>(x0, d.T, lmed, warp, stage, base);
    else if (d.m <= 32)
        summarise_steps<1>(x0, d.T, d.m, lmed, warp, base);
    else if (d.m <= 64)
        summarise_steps<2>(x0, d.T, d.m, lmed, warp, base);
    else if (d.m <= 128)
        summarise_steps<4>(x0, d.T, d.m, lmed, warp, base);
    else
        summarise_steps<8>(x0, d.T, d.m, lmed, warp, base);
}

}  // namespace

cudaError_t launch_summaries(const uint32_t *samples, const SeriesDesc *raw_desc, int64_t S, uint16_t *feat,
                             cudaStream_t st, const unsigned long long *gate) {
    if (S <= 0) return cudaSuccess;
    static int configured_device = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_device != dev) {
        e = cudaFuncSetAttribute(summaries_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSumSmem);
        if (e != cudaSuccess) return e;
        configured_device = dev;
    }
    summaries_kernel<<<(unsigned)S, kSumWarps * 32, kSumSmem, st>>>(samples, raw_desc,
                                                                   reinterpret_cast<__nv_bfloat16 *>(feat), gate);
    return cudaGetLastError();
}

}  // namespace mt4g
