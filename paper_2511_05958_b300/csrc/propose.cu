// Change-point windows from the proposal network's per-step logits.
//
// For each series: softmax over its T steps; repeatedly take the largest remaining logit
// (smallest step on ties) as a window centre c and remove the steps within +-half of it,
// n_win times; conf = softmax mass of the union of the windows [c - half, c + half].
#include "mt4g_cnn.cuh"

namespace mt4g {

namespace {

__global__ void __launch_bounds__(256) propose_kernel(const float *__restrict__ logits,
                                                      const SeriesDesc *__restrict__ desc, int32_t n_win,
                                                      int32_t half, int32_t *__restrict__ win_center,
                                                      float *__restrict__ conf,
                                                      const unsigned long long *__restrict__ gate) {
    if (gate && *gate == 0ull) return;
    __shared__ float s_v[8];
    __shared__ int s_i[8];
    __shared__ float s_max, s_sum;
    __shared__ int s_c;
    const int64_t s = blockIdx.x;
    const SeriesDesc d = desc[s];
    const float *z = logits + row_base(d, s) + 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // softmax normaliser
    float mx = -INFINITY;
    for (int t = tid; t < d.T; t += 256) mx = fmaxf(mx, z[t]);
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) s_v[warp] = mx;
    __syncthreads();
    if (tid == 0) {
        float v = s_v[0];
        for (int w = 1; w < 8; w++) v = fmaxf(v, s_v[w]);
        s_max = v;
    }
    __syncthreads();
    float sum = 0.f;
    for (int t = tid; t < d.T; t += 256) sum += expf(z[t] - s_max);
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) s_v[warp] = sum;
    __syncthreads();
    if (tid == 0) {
        float v = 0.f;
        for (int w = 0; w < 8; w++) v += s_v[w];
        s_sum = v;
    }
    __syncthreads();
    // greedy windows; a step is alive while no chosen window covers it
    float covered = 0.f;
    int centres[8];
    int nc = 0;
    for (int w = 0; w < n_win; w++) {
        float bv = -INFINITY;
        int bi = 0x7fffffff;
        for (int t = tid; t < d.T; t += 256) {
            bool alive = true;
            for (int c = 0; c < nc; c++) alive &= (t < centres[c] - half || t > centres[c] + half);
            const float v = z[t];
            if (alive && (v > bv || (v == bv && t < bi))) {
                bv = v;
                bi = t;
            }
        }
        for (int o = 16; o; o >>= 1) {
            const float v2 = __shfl_xor_sync(0xffffffffu, bv, o);
            const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
            if (v2 > bv || (v2 == bv && i2 < bi)) {
                bv = v2;
                bi = i2;
            }
        }
        __syncthreads();
        if (lane == 0) {
            s_v[warp] = bv;
            s_i[warp] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            float v = s_v[0];
            int i = s_i[0];
            for (int q = 1; q < 8; q++)
                if (s_v[q] > v || (s_v[q] == v && s_i[q] < i)) {
                    v = s_v[q];
                    i = s_i[q];
                }
            s_c = (i == 0x7fffffff) ? -1 : i;
        }
        __syncthreads();
        const int c = s_c;
        if (c < 0) break;
        centres[nc++] = c;
        if (tid == 0) win_center[s * n_win + w] = c;
    }
    if (tid == 0)
        for (int w = nc; w < n_win; w++) win_center[s * n_win + w] = -1;
    for (int t = tid; t < d.T; t += 256) {
        bool in = false;
        for (int c = 0; c < nc; c++) in |= (t >= centres[c] - half && t <= centres[c] + half);
        if (in) covered += expf(z[t] - s_max);
    }
    for (int o = 16; o; o >>= 1) covered += __shfl_xor_sync(0xffffffffu, covered, o);
    __syncthreads();
    if (lane == 0) s_v[warp] = covered;
    __syncthreads();
    if (tid == 0) {
        float v = 0.f;
        for (int w = 0; w < 8; w++) v += s_v[w];
        conf[s] = v / s_sum;
    }
}

}  // namespace

cudaError_t launch_propose(const float *logits, const SeriesDesc *desc, int64_t S, int32_t n_win, int32_t half,
                           int32_t *win_center, float *conf, cudaStream_t st, const unsigned long long *gate) {
    if (S <= 0) return cudaSuccess;
    propose_kernel<<<(unsigned)S, 256, 0, st>>>(logits, desc, n_win, half, win_center, conf, gate);
    return cudaGetLastError();
}

}  // namespace mt4g

namespace mt4g {
namespace {
__global__ void zero_pad_rows_kernel(uint8_t *buf, int row_bytes, const SeriesDesc *__restrict__ desc, int64_t S) {
    const int64_t s = blockIdx.x;
    const SeriesDesc d = desc[s];
    const int64_t r0 = row_base(d, s);
    for (int e = threadIdx.x; e < 4 * row_bytes; e += blockDim.x) {
        const int r = e / row_bytes, c = e % row_bytes;
        const int64_t row = r < 2 ? r0 + r : r0 + d.T + r;  // rows 0, 1 and T + 2, T + 3
        buf[row * row_bytes + c] = 0;
    }
}
}  // namespace

cudaError_t launch_zero_pad_rows(void *buf, int row_bytes, const SeriesDesc *desc, int64_t S, cudaStream_t st) {
    if (S <= 0 || !buf) return cudaSuccess;
    zero_pad_rows_kernel<<<(unsigned)S, 128, 0, st>>>((uint8_t *)buf, row_bytes, desc, S);
    return cudaGetLastError();
}
}  // namespace mt4g
