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
// One warp per step: the step's m <= 256 samples are sorted in registers by a bitonic
// network (V values per lane, partners across lanes by shuffle), then lanes 0..15 pick
// their quantile.  Each warp takes every eighth step and loads the next one while sorting.
#include <cuda_bf16.h>

#include "mt4g_internal.cuh"

namespace mt4g {

namespace {

constexpr unsigned kFull = 0xffffffffu;

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

// Features of steps warp, warp + 8, ... of one series; each step's samples are loaded one
// step ahead, so the loads of the next step are in flight while this one is sorted.
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
    for (int t = warp; t < T; t += 8) {
        uint32_t x[V];
#pragma unroll
        for (int r = 0; r < V; r++) x[r] = nx[r];
        if (t + 8 < T) load(t + 8, nx);
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

__global__ void __launch_bounds__(256, 4) summaries_kernel(const uint32_t *__restrict__ samples,
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
    if (d.m <= 32)
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
    summaries_kernel<<<(unsigned)S, 256, 0, st>>>(samples, raw_desc, reinterpret_cast<__nv_bfloat16 *>(feat), gate);
    return cudaGetLastError();
}

}  // namespace mt4g
