// Load-latency statistics per series (paper Sec. IV-C: the average as the main result,
// with p50, p95 and the standard deviation), over all T*m samples of a series.
//
//   mean = (sum x) / N: the exact 64-bit integer sum rounded once to FP64, one division;
//   p50, p95: nearest-rank order statistics sorted[ceil(q N) - 1], read from the sorted
//       keys by the sort kernel (SeriesDesc::p50 / p95);
//   std = sqrt(var), var = (N sum x^2 - (sum x)^2) / N^2 (population variance), with the
//       numerator exact in 128-bit integers, rounded once to FP64 (nearest, ties to even),
//       divided by the FP64 product N * N.
// Every rounding is an explicit IEEE round-to-nearest step, so the results are the same
// bits a plain host evaluation of these formulas gives.  One CTA per series streams its
// samples once (4 B per sample: HBM-bound).
#include "mt4g_internal.cuh"

namespace mt4g {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kStatsThreads = 256;

// (hi, lo) += (h2, l2) on 128-bit unsigned values.
__device__ __forceinline__ void add128(uint64_t &hi, uint64_t &lo, uint64_t h2, uint64_t l2) {
    lo += l2;
    hi += h2 + (lo < l2 ? 1u : 0u);
}

// 128-bit unsigned value hi * 2^64 + lo rounded to the nearest double, ties to even.
__device__ double u128_to_double_rn(uint64_t hi, uint64_t lo) {
    if (hi == 0) return __ull2double_rn(lo);
    const int sh = 64 - __clzll((long long)hi);  // bits of hi, 1..64; the value has 64 + sh bits
    // the top 64 bits of the value, and whether any bit below them is set
    const uint64_t top = sh == 64 ? hi : ((hi << (64 - sh)) | (lo >> sh));
    const bool sticky = sh == 64 ? lo != 0 : (lo << (64 - sh)) != 0;
    uint64_t mant = top >> 11;  // 53 bits with the leading one
    const uint64_t rem = top & 0x7ffu;
    if (rem > 0x400u || (rem == 0x400u && (sticky || (mant & 1u)))) mant++;
    return ldexp((double)mant, 11 + sh);  // exact: mant <= 2^53, a power-of-two scale
}

__global__ void __launch_bounds__(kStatsThreads) latency_stats_kernel(const uint32_t *__restrict__ samples,
                                                                      const SeriesDesc *__restrict__ desc,
                                                                      double *mean_out, uint32_t *p50_out,
                                                                      uint32_t *p95_out, double *std_out) {
    __shared__ uint64_t s_sum[kStatsThreads / 32], s_hi[kStatsThreads / 32], s_lo[kStatsThreads / 32];
    const int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const SeriesDesc d = desc[s];
    const int64_t N = (int64_t)d.T * d.m;
    const uint32_t *x = samples + d.off;
    uint64_t sx = 0, qhi = 0, qlo = 0;
    for (int64_t i = tid; i < N; i += kStatsThreads) {
        const uint64_t v = __ldg(x + i);
        sx += v;
        add128(qhi, qlo, 0, v * v);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        sx += __shfl_xor_sync(kFull, sx, o);
        const uint64_t h2 = __shfl_xor_sync(kFull, qhi, o), l2 = __shfl_xor_sync(kFull, qlo, o);
        add128(qhi, qlo, h2, l2);
    }
    if (lane == 0) {
        s_sum[warp] = sx;
        s_hi[warp] = qhi;
        s_lo[warp] = qlo;
    }
    __syncthreads();
    if (tid != 0) return;
    sx = 0;
    qhi = 0;
    qlo = 0;
    for (int w = 0; w < kStatsThreads / 32; w++) {
        sx += s_sum[w];
        add128(qhi, qlo, s_hi[w], s_lo[w]);
    }
    // N sum x^2 - (sum x)^2 in 128 bits (N < 2^31, sum x^2 < 2^95, sum x < 2^63)
    const uint64_t n = (uint64_t)N;
    uint64_t ahi = __umul64hi(n, qlo) + n * qhi, alo = n * qlo;
    const uint64_t bhi = __umul64hi(sx, sx), blo = sx * sx;
    const uint64_t borrow = alo < blo ? 1u : 0u;
    alo -= blo;
    ahi = ahi - bhi - borrow;
    const double dn = (double)N;
    mean_out[s] = __ddiv_rn(__ull2double_rn(sx), dn);
    std_out[s] = __dsqrt_rn(__ddiv_rn(u128_to_double_rn(ahi, alo), __dmul_rn(dn, dn)));
    p50_out[s] = d.p50;
    p95_out[s] = d.p95;
}

}  // namespace

cudaError_t launch_latency_stats(const uint32_t *samples, const SeriesDesc *desc, int64_t S, double *mean_out,
                                 uint32_t *p50_out, uint32_t *p95_out, double *std_out, cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    latency_stats_kernel<<<(unsigned)S, kStatsThreads, 0, st>>>(samples, desc, mean_out, p50_out, p95_out, std_out);
    return cudaGetLastError();
}

}  // namespace mt4g
