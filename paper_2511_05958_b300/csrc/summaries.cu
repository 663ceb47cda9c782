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
// their quantile.
#include <cuda_bf16.h>

#include "mt4g_internal.cuh"

namespace mt4g {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// Ascending bitonic sort of 32 V values; lane l holds elements l V .. l V + V - 1.
template <int V>
__device__ __forceinline__ void bitonic_sort_warp(uint32_t (&x)[V]) {
    const int lane = threadIdx.x & 31;
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
                        const bool up = ((lane * V + r) & k) == 0;
                        const uint32_t a = x[r], b = x[p];
                        if ((a > b) == up) {
                            x[r] = b;
                            x[p] = a;
                        }
                    }
                }
            } else {
                const int lj = j / V;
#pragma unroll
                for (int r = 0; r < V; r++) {
                    const int e = lane * V + r;
                    const uint32_t o = __shfl_xor_sync(kFull, x[r], lj);
                    const bool up = (e & k) == 0;
                    const bool lower = (e & j) == 0;
                    x[r] = (lower == up) ? min(x[r], o) : max(x[r], o);
                }
            }
        }
    }
}

template <int V>
__device__ void summarise_step(const uint32_t *__restrict__ row, int m, float lmed, int t,
                               __nv_bfloat16 *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    uint32_t x[V];
#pragma unroll
    for (int r = 0; r < V; r++) {
        const int e = lane * V + r;
        x[r] = e < m ? __ldg(row + e) : 0xffffffffu;
    }
    bitonic_sort_warp<V>(x);
    const int i = lane & 15;
    const int rank = min(m - 1, ((2 * i + 1) * m) / 32);
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
    if (lane < kFeatC) out[lane] = __float2bfloat16_rn(f);
}

__global__ void __launch_bounds__(256, 4) summaries_kernel(const uint32_t *__restrict__ samples,
                                                        const SeriesDesc *__restrict__ desc,
                                                        __nv_bfloat16 *__restrict__ feat) {
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
    for (int t = warp; t < d.T; t += 8) {
        const uint32_t *row = samples + d.off + (int64_t)t * d.m;
        __nv_bfloat16 *out = base + (int64_t)(2 + t) * kFeatC;
        if (d.m <= 32)
            summarise_step<1>(row, d.m, lmed, t, out);
        else if (d.m <= 64)
            summarise_step<2>(row, d.m, lmed, t, out);
        else if (d.m <= 128)
            summarise_step<4>(row, d.m, lmed, t, out);
        else
            summarise_step<8>(row, d.m, lmed, t, out);
    }
}

}  // namespace

cudaError_t launch_summaries(const uint32_t *samples, const SeriesDesc *raw_desc, int64_t S, uint16_t *feat,
                             cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    summaries_kernel<<<(unsigned)S, 256, 0, st>>>(samples, raw_desc, reinterpret_cast<__nv_bfloat16 *>(feat));
    return cudaGetLastError();
}

}  // namespace mt4g
