// The change-point proposal network and its training kernels.
//
// The paper scans every index (Sec. IV-B-1 (4)) and mentions shortlisting candidate
// change points to save computation (Sec. IV-B-1, after (4)).  The shortlist here comes
// from a small 1D CNN over the per-step summaries: four width-5 convolutions along the
// step axis (zero padding 2), 18 (17 + a zero channel) -> 32 -> 32 -> 32 -> 1 channels,
// ReLU after the first three, one logit per step.
//
// Precision: inputs, hidden activations and the weights used by the kernels are BF16
// (weights are the BF16 rounding of FP32 master weights; biases stay FP32); every sum
// accumulates in FP32 (weight gradients: FP32 per tile, FP64 across tiles); logits,
// gradients and the Adam state are FP32.
//
// Layout: activations are [rows][C] with the padded row layout of the summaries (two zero
// rows on each side of every series), so a window of 5 steps is 5 consecutive rows.
// Weights of a layer are stored [5][Cin][Cout] (tap-major, output channel fastest).
// Training batches have one T for all series.
//
// Loss: softmax over a series' T steps, cross-entropy against the distribution uniform
// over its change points; series without change points are left out; the mean is over
// the series that carry a target.  Adam (Kingma & Ba) with bias correction.
#include <cuda_bf16.h>

#include <vector>

#include "mt4g_cnn.cuh"

namespace mt4g {

namespace {

constexpr int kTile = 128;  // positions per block

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

// Position tile -> (series, first step).  tiles_before[s] = tiles of series < s.
__device__ __forceinline__ int64_t find_series(const int64_t *__restrict__ tiles_before, int64_t S, int64_t tile) {
    int64_t lo = 0, hi = S - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (tiles_before[mid] <= tile)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// out[pos][o] = b[o] + sum_{d,i} W[d][i][o] in[pos + d - 2][i], over a tile of 64 positions
// and all 32 outputs.  HIDDEN: ReLU and BF16 store.  MASKED (backward data pass): the input
// is an FP32 gradient, W is the flipped transpose, and the result is multiplied by the
// mask (act > 0) and stored FP32 without bias.
template <int CIN, typename TIn, bool BWD>
__global__ void __launch_bounds__(128) conv32_kernel(const TIn *__restrict__ in, const float *__restrict__ W,
                                                     const float *__restrict__ bias, void *__restrict__ out,
                                                     const __nv_bfloat16 *__restrict__ mask_act,
                                                     const SeriesDesc *__restrict__ desc,
                                                     const int64_t *__restrict__ tiles_before, int64_t S) {
    constexpr int kP = 4;  // positions per thread (consecutive)
    __shared__ float xs[kTile + 4][CIN + 1];
    __shared__ __align__(16) float ws[5 * CIN][32];
    const int64_t tile = blockIdx.x;
    const int64_t s = find_series(tiles_before, S, tile);
    const SeriesDesc d = desc[s];
    const int t0 = (int)(tile - tiles_before[s]) * kTile;
    const int64_t r0 = row_base(d, s) + t0;  // padded row of the window start of position t0
    const int nrows = min(kTile + 4, d.T + 4 - t0);
    for (int e = threadIdx.x; e < (kTile + 4) * CIN; e += 128) {
        const int r = e / CIN, c = e % CIN;
        float v = 0.f;
        if (r < nrows) {
            if constexpr (sizeof(TIn) == 2)
                v = bf(in[(r0 + r) * CIN + c]);
            else
                v = in[(r0 + r) * CIN + c];
        }
        xs[r][c] = v;
    }
    for (int e = threadIdx.x; e < 5 * CIN * 32; e += 128) ws[e / 32][e % 32] = W[e];
    __syncthreads();
    const int p0 = (threadIdx.x >> 2) * kP, og = threadIdx.x & 3;
    float acc[kP][8];
#pragma unroll
    for (int q = 0; q < kP; q++)
#pragma unroll
        for (int j = 0; j < 8; j++) acc[q][j] = BWD ? 0.f : bias[og * 8 + j];
#pragma unroll
    for (int dd = 0; dd < 5; dd++) {
#pragma unroll 2
        for (int i = 0; i < CIN; i++) {
            const float4 w0 = *reinterpret_cast<const float4 *>(&ws[dd * CIN + i][og * 8]);
            const float4 w1 = *reinterpret_cast<const float4 *>(&ws[dd * CIN + i][og * 8 + 4]);
#pragma unroll
            for (int q = 0; q < kP; q++) {
                const float x = xs[p0 + q + dd][i];
                acc[q][0] = fmaf(x, w0.x, acc[q][0]);
                acc[q][1] = fmaf(x, w0.y, acc[q][1]);
                acc[q][2] = fmaf(x, w0.z, acc[q][2]);
                acc[q][3] = fmaf(x, w0.w, acc[q][3]);
                acc[q][4] = fmaf(x, w1.x, acc[q][4]);
                acc[q][5] = fmaf(x, w1.y, acc[q][5]);
                acc[q][6] = fmaf(x, w1.z, acc[q][6]);
                acc[q][7] = fmaf(x, w1.w, acc[q][7]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kP; q++) {
        if (t0 + p0 + q >= d.T) break;
        const int64_t row = r0 + 2 + p0 + q;
        if (!BWD) {
            __nv_bfloat162 *o = reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<__nv_bfloat16 *>(out) + row * 32 + og * 8);
#pragma unroll
            for (int j = 0; j < 4; j++)
                o[j] = __floats2bfloat162_rn(fmaxf(acc[q][2 * j], 0.f), fmaxf(acc[q][2 * j + 1], 0.f));
        } else {
            float *o = reinterpret_cast<float *>(out) + row * 32 + og * 8;
            const __nv_bfloat16 *ma = mask_act + row * 32 + og * 8;
#pragma unroll
            for (int j = 0; j < 8; j++) o[j] = bf(ma[j]) > 0.f ? acc[q][j] : 0.f;
        }
    }
}

// Last layer, 32 -> 1: logits[row] = b + sum_{d,i} W4[d][i] a3[row + d - 2][i].  The tile's
// kTile + 4 activation rows (64 B each) are staged in shared memory with 16-byte loads first, so
// every row is read from memory once.
__global__ void __launch_bounds__(kTile) conv_out_kernel(const __nv_bfloat16 *__restrict__ a3,
                                                         const float *__restrict__ W4, const float *__restrict__ b4,
                                                         float *__restrict__ logits,
                                                         const SeriesDesc *__restrict__ desc,
                                                         const int64_t *__restrict__ tiles_before, int64_t S,
                                                         const unsigned long long *__restrict__ gate) {
    if (gate && *gate == 0ull) return;
    __shared__ float w[5 * 32];
    __shared__ __align__(16) uint4 xs[(kTile + 4) * 4];  // 8 BF16 channels per uint4
    const int64_t tile = blockIdx.x;
    const int64_t s = find_series(tiles_before, S, tile);
    const SeriesDesc d = desc[s];
    const int t0 = (int)(tile - tiles_before[s]) * kTile;
    const int64_t r0 = row_base(d, s) + t0;  // padded row of the window start of position t0
    const int nrows = min(kTile + 4, d.T + 4 - t0);
    const uint4 *src = reinterpret_cast<const uint4 *>(a3 + r0 * 32);
    for (int e = threadIdx.x; e < (kTile + 4) * 4; e += kTile) xs[e] = e < nrows * 4 ? src[e] : make_uint4(0, 0, 0, 0);
    for (int e = threadIdx.x; e < 160; e += kTile) w[e] = W4[e];
    __syncthreads();
    const int t = t0 + threadIdx.x;
    if (t >= d.T) return;
    float acc = b4[0];
#pragma unroll
    for (int dd = 0; dd < 5; dd++) {
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const uint4 v = xs[(threadIdx.x + dd) * 4 + c];
            const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int h = 0; h < 4; h++) {
                const float lo = __uint_as_float(u[h] << 16), hi = __uint_as_float(u[h] & 0xffff0000u);
                acc = fmaf(lo, w[dd * 32 + c * 8 + 2 * h], acc);
                acc = fmaf(hi, w[dd * 32 + c * 8 + 2 * h + 1], acc);
            }
        }
    }
    logits[r0 + 2 + threadIdx.x] = acc;
}

// dA3[row][i] = [a3 > 0] sum_d W4[d][i] g[row + 2 - d]  (gradient through the last layer)
__global__ void __launch_bounds__(256) bwd_out_kernel(const float *__restrict__ g, const float *__restrict__ W4,
                                                      const __nv_bfloat16 *__restrict__ a3, float *__restrict__ dz3,
                                                      const SeriesDesc *__restrict__ desc, int64_t S, int T) {
    const int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x;  // (series, t, i)
    const int64_t total = S * (int64_t)T * 32;
    if (e >= total) return;
    const int i = (int)(e & 31);
    const int64_t st = e >> 5;
    const int64_t s = st / T;
    const int t = (int)(st % T);
    const int64_t row = row_base(desc[s], s) + 2 + t;
    float acc = 0.f;
#pragma unroll
    for (int dd = 0; dd < 5; dd++) acc = fmaf(W4[dd * 32 + i], g[row + 2 - dd], acc);
    dz3[row * 32 + i] = bf(a3[row * 32 + i]) > 0.f ? acc : 0.f;
}

// dW[d][i][o] += sum_pos dz[pos][o] a[pos + d - 2][i];  db[o] += sum_pos dz[pos][o].
// A block reduces `tiles_per_block` tiles of one batch (uniform T) before one atomicAdd per
// weight.  COUT = 32 (hidden layers) or 1 (last layer, dz = g as [rows][1]).
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) wgrad_kernel(const float *__restrict__ dz, const __nv_bfloat16 *__restrict__ a,
                                                    double *__restrict__ dW, double *__restrict__ db,
                                                    const SeriesDesc *__restrict__ desc, int64_t S, int T,
                                                    int tiles_per_series, int tiles_per_block) {
    constexpr int KK = 5 * CIN;
    constexpr int NACC = (KK * COUT + 255) / 256;
    __shared__ float zs[kTile][COUT];
    __shared__ float as[kTile + 4][CIN + 1];
    double acc[NACC];
    double bacc = 0.0;
#pragma unroll
    for (int j = 0; j < NACC; j++) acc[j] = 0.0;
    const int64_t ntiles = S * tiles_per_series;
    for (int64_t tile = (int64_t)blockIdx.x * tiles_per_block;
         tile < min(ntiles, (int64_t)(blockIdx.x + 1) * tiles_per_block); tile++) {
        const int64_t s = tile / tiles_per_series;
        const int t0 = (int)(tile % tiles_per_series) * kTile;
        const int64_t r0 = row_base(desc[s], s) + t0;
        const int npos = min(kTile, T - t0);
        __syncthreads();
        for (int e = threadIdx.x; e < kTile * COUT; e += 256) {
            const int p = e / COUT, o = e % COUT;
            zs[p][o] = p < npos ? dz[(r0 + 2 + p) * COUT + o] : 0.f;
        }
        for (int e = threadIdx.x; e < (kTile + 4) * CIN; e += 256) {
            const int r = e / CIN, c = e % CIN;
            as[r][c] = r < npos + 4 ? bf(a[(r0 + r) * CIN + c]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < NACC; j++) {
            const int w = threadIdx.x + 256 * j;
            if (w < KK * COUT) {
                const int o = w % COUT, kk = w / COUT;
                const int dd = kk / CIN, i = kk % CIN;
                float s0 = 0.f, s1 = 0.f;  // two chains: shorter fp32 sums per tile
                for (int p = 0; p < kTile; p += 2) {
                    s0 = fmaf(zs[p][o], as[p + dd][i], s0);
                    s1 = fmaf(zs[p + 1][o], as[p + 1 + dd][i], s1);
                }
                acc[j] += (double)s0 + (double)s1;
            }
        }
        if (threadIdx.x < COUT) {
            float sb = 0.f;
            for (int p = 0; p < kTile; p++) sb += zs[p][threadIdx.x];
            bacc += (double)sb;
        }
    }
#pragma unroll
    for (int j = 0; j < NACC; j++) {
        const int w = threadIdx.x + 256 * j;
        if (w < KK * COUT) atomicAdd(dW + w, acc[j]);
    }
    if (threadIdx.x < COUT) atomicAdd(db + threadIdx.x, bacc);
}

// Gradients accumulate in FP64 across tiles (the softmax gradient sums to zero over the
// steps, so the weight sums cancel heavily); this writes them back as FP32.
__global__ void grad_to_float_kernel(const double *__restrict__ gd, float *__restrict__ g) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < kCnnParams) g[e] = (float)gd[e];
}

// Softmax over the T steps of each series and the cross-entropy gradient
// g = (p - y) / n_valid, y uniform over the series' change points.
__global__ void __launch_bounds__(256) softmax_ce_kernel(const float *__restrict__ logits, float *__restrict__ g,
                                                         const int32_t *__restrict__ cp_count,
                                                         const int32_t *__restrict__ cp_idx, int32_t max_cp,
                                                         const SeriesDesc *__restrict__ desc, int T,
                                                         const float *__restrict__ inv_valid, float *loss) {
    __shared__ float red[8];
    __shared__ float s_max, s_sum;
    const int64_t s = blockIdx.x;
    const int64_t rb = row_base(desc[s], s) + 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int nc = min(cp_count[s], max_cp);
    float mx = -INFINITY;
    for (int t = tid; t < T; t += 256) mx = fmaxf(mx, logits[rb + t]);
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    if (tid == 0) {
        float v = red[0];
        for (int w = 1; w < 8; w++) v = fmaxf(v, red[w]);
        s_max = v;
    }
    __syncthreads();
    float sum = 0.f;
    for (int t = tid; t < T; t += 256) sum += expf(logits[rb + t] - s_max);
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    __syncthreads();
    if (lane == 0) red[warp] = sum;
    __syncthreads();
    if (tid == 0) {
        float v = 0.f;
        for (int w = 0; w < 8; w++) v += red[w];
        s_sum = v;
    }
    __syncthreads();
    const float scale = nc > 0 ? inv_valid[0] : 0.f;
    const float lse = s_max + logf(s_sum);
    for (int t = tid; t < T; t += 256) {
        const float p = expf(logits[rb + t] - lse);
        float y = 0.f;
        for (int c = 0; c < nc; c++) y += (cp_idx[s * max_cp + c] == t) ? 1.f / (float)nc : 0.f;
        g[rb + t] = (p - y) * scale;
    }
    if (tid == 0 && nc > 0) {
        float l = 0.f;
        for (int c = 0; c < nc; c++) l += lse - logits[rb + cp_idx[s * max_cp + c]];
        atomicAdd(loss, l / (float)nc * scale);
    }
}

// 1 / (number of series with at least one change point), for the mean loss.
__global__ void count_valid_kernel(const int32_t *__restrict__ cp_count, int64_t S, float *inv_valid) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    int c = 0;
    for (int64_t s = threadIdx.x; s < S; s += blockDim.x) c += cp_count[s] > 0;
    atomicAdd(&cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) inv_valid[0] = cnt > 0 ? 1.f / (float)cnt : 0.f;
}

// Weights used by the kernels: BF16 rounding of the masters, and the flipped transposes
// for the backward data pass: Wt[d'][o][i] = W[4 - d'][i][o].
__global__ void prepare_weights_kernel(const float *__restrict__ master, float *__restrict__ used,
                                       float *__restrict__ flipped) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < kCnnParams) {
        // weights are read as BF16; biases stay FP32
        const bool bias = (e >= cnn_off(1) && e < cnn_off(2)) || (e >= cnn_off(3) && e < cnn_off(4)) ||
                          (e >= cnn_off(5) && e < cnn_off(6)) || e >= cnn_off(7);
        used[e] = bias ? master[e] : __bfloat162float(__float2bfloat16_rn(master[e]));
    }
    // flipped transposes of layers 2 and 3 (and 1 is never needed)
    for (int l = 1; l <= 2; l++) {
        const int off = cnn_off(2 * l);
        if (e < 5 * 32 * 32) {
            const int dd = e / 1024, rem = e % 1024, o = rem / 32, i = rem % 32;
            const int src = off + ((4 - dd) * 32 + i) * 32 + o;
            flipped[(l - 1) * 5120 + e] = __bfloat162float(__float2bfloat16_rn(master[src]));
        }
    }
}

__global__ void adam_kernel(float *__restrict__ master, const float *__restrict__ grad, float *__restrict__ m1,
                            float *__restrict__ m2, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kCnnParams) return;
    const float g = grad[e];
    const float m = b1 * m1[e] + (1.f - b1) * g;
    const float v = b2 * m2[e] + (1.f - b2) * g * g;
    m1[e] = m;
    m2[e] = v;
    const float mh = m / c1, vh = v / c2;
    master[e] -= lr * mh / (sqrtf(vh) + eps);
}

}  // namespace

// ---------------------------------------------------------------- host-side launchers

int64_t cnn_tiles(const std::vector<SeriesDesc> &desc, std::vector<int64_t> &tiles_before) {
    tiles_before.resize(desc.size());
    int64_t n = 0;
    for (size_t s = 0; s < desc.size(); s++) {
        tiles_before[s] = n;
        n += (desc[s].T + kTile - 1) / kTile;
    }
    return n;
}

cudaError_t cnn_prepare(const CnnState &W, cudaStream_t st) {
    prepare_weights_kernel<<<(kCnnParams + 255) / 256, 256, 0, st>>>(W.master, W.used, W.flipped);
    return cudaGetLastError();
}

cudaError_t cnn_forward(const CnnState &W, const uint16_t *feat, const CnnActs &A, const SeriesDesc *desc,
                        const int64_t *tiles_before, int64_t S, int64_t ntiles, long long wait_limit_ns,
                        int32_t *status, cudaStream_t st, const unsigned long long *gate) {
    if (ntiles <= 0) return cudaSuccess;
    const __nv_bfloat16 *x0 = reinterpret_cast<const __nv_bfloat16 *>(feat);
    const float *u = W.used;
    // the three hidden layers on the tensor cores (conv_tc.cu), the 32 -> 1 layer below
    __nv_bfloat16 *a1 = reinterpret_cast<__nv_bfloat16 *>(A.a1), *a2 = reinterpret_cast<__nv_bfloat16 *>(A.a2),
                  *a3 = reinterpret_cast<__nv_bfloat16 *>(A.a3);
    cudaError_t e = cnn_hidden_tc(0, x0, u + cnn_off(0), u + cnn_off(1), a1, desc, tiles_before, S, ntiles,
                                  wait_limit_ns, status, st, gate);
    if (e == cudaSuccess)
        e = cnn_hidden_tc(1, a1, u + cnn_off(2), u + cnn_off(3), a2, desc, tiles_before, S, ntiles, wait_limit_ns,
                          status, st, gate);
    if (e == cudaSuccess)
        e = cnn_hidden_tc(2, a2, u + cnn_off(4), u + cnn_off(5), a3, desc, tiles_before, S, ntiles, wait_limit_ns,
                          status, st, gate);
    if (e != cudaSuccess) return e;
    conv_out_kernel<<<(unsigned)ntiles, kTile, 0, st>>>(reinterpret_cast<const __nv_bfloat16 *>(A.a3),
                                                        u + cnn_off(6), u + cnn_off(7), A.logits, desc, tiles_before, S,
                                                        gate);
    return cudaGetLastError();
}

cudaError_t cnn_backward(const CnnState &W, const uint16_t *feat, const CnnActs &A, const int32_t *cp_count,
                         const int32_t *cp_idx, int32_t max_cp, const SeriesDesc *desc, int64_t S, int T,
                         float *grad, float *loss, cudaStream_t st) {
    const int tps = (T + kTile - 1) / kTile;
    const int64_t ntiles = S * tps;
    const int tpb = 16;
    const unsigned wblocks = (unsigned)((ntiles + tpb - 1) / tpb);
    double *gd = W.grad64;
    cudaMemsetAsync(gd, 0, kCnnParams * sizeof(double), st);
    cudaMemsetAsync(loss, 0, sizeof(float), st);
    count_valid_kernel<<<1, 256, 0, st>>>(cp_count, S, A.inv_valid);
    softmax_ce_kernel<<<(unsigned)S, 256, 0, st>>>(A.logits, A.g, cp_count, cp_idx, max_cp, desc, T, A.inv_valid,
                                                     loss);
    const float *u = W.used;
    const __nv_bfloat16 *a1 = reinterpret_cast<const __nv_bfloat16 *>(A.a1);
    const __nv_bfloat16 *a2 = reinterpret_cast<const __nv_bfloat16 *>(A.a2);
    const __nv_bfloat16 *a3 = reinterpret_cast<const __nv_bfloat16 *>(A.a3);
    const __nv_bfloat16 *x0 = reinterpret_cast<const __nv_bfloat16 *>(feat);
    // layer 4
    wgrad_kernel<32, 1><<<wblocks, 256, 0, st>>>(A.g, a3, gd + cnn_off(6), gd + cnn_off(7), desc, S, T, tps, tpb);
    const int64_t n3 = S * (int64_t)T * 32;
    bwd_out_kernel<<<(unsigned)((n3 + 255) / 256), 256, 0, st>>>(A.g, u + cnn_off(6), a3, A.dz3, desc, S, T);
    // layer 3
    wgrad_kernel<32, 32><<<wblocks, 256, 0, st>>>(A.dz3, a2, gd + cnn_off(4), gd + cnn_off(5), desc, S, T, tps, tpb);
    conv32_kernel<32, float, true><<<(unsigned)ntiles, 128, 0, st>>>(A.dz3, W.flipped + 5120, nullptr, A.dz2, a2, desc,
                                                                     A.tiles_before, S);
    // layer 2
    wgrad_kernel<32, 32><<<wblocks, 256, 0, st>>>(A.dz2, a1, gd + cnn_off(2), gd + cnn_off(3), desc, S, T, tps, tpb);
    conv32_kernel<32, float, true><<<(unsigned)ntiles, 128, 0, st>>>(A.dz2, W.flipped, nullptr, A.dz1, a1, desc,
                                                                     A.tiles_before, S);
    // layer 1
    wgrad_kernel<kFeatC, 32><<<wblocks, 256, 0, st>>>(A.dz1, x0, gd + cnn_off(0), gd + cnn_off(1), desc, S, T, tps,
                                                      tpb);
    grad_to_float_kernel<<<(kCnnParams + 255) / 256, 256, 0, st>>>(gd, grad);
    return cudaGetLastError();
}

cudaError_t cnn_adam(CnnState &W, const float *grad, float lr, cudaStream_t st) {
    W.step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)W.step), c2 = 1.f - powf(b2, (float)W.step);
    adam_kernel<<<(kCnnParams + 255) / 256, 256, 0, st>>>(W.master, grad, W.m1, W.m2, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

}  // namespace mt4g
