// Proposal network: parameter layout, device state and launchers (see cnn.cu).
#pragma once
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "mt4g_internal.cuh"

namespace mt4g {

// Flat FP32 parameter vector: W1 [5][18][32], b1 [32], W2 [5][32][32], b2 [32],
// W3 [5][32][32], b3 [32], W4 [5][32][1], b4 [1].  Input channel 17 of W1 multiplies a
// zero feature, so the 160 weights on it never change.
constexpr int kCnnParams = 5 * kFeatC * 32 + 32 + 2 * (5 * 32 * 32 + 32) + 5 * 32 + 1;
__host__ __device__ constexpr int cnn_off(int i) {
    return i == 0   ? 0
           : i == 1 ? 5 * kFeatC * 32
           : i == 2 ? 5 * kFeatC * 32 + 32
           : i == 3 ? 5 * kFeatC * 32 + 32 + 5120
           : i == 4 ? 5 * kFeatC * 32 + 32 + 5152
           : i == 5 ? 5 * kFeatC * 32 + 32 + 5152 + 5120
           : i == 6 ? 5 * kFeatC * 32 + 32 + 2 * 5152
                    : 5 * kFeatC * 32 + 32 + 2 * 5152 + 160;
}

struct CnnState {
    float *master = nullptr;   // FP32 master weights [kCnnParams]
    float *used = nullptr;     // BF16-rounded copy the kernels read
    float *flipped = nullptr;  // flipped transposes of W2, W3 for the backward data pass [2][5][32][32]
    float *m1 = nullptr;       // Adam first moment
    float *m2 = nullptr;       // Adam second moment
    float *grad = nullptr;     // gradient scratch
    double *grad64 = nullptr;  // FP64 accumulation of the gradients
    float *loss = nullptr;     // device scalar
    long long step = 0;        // Adam steps taken
};

struct CnnActs {
    uint16_t *a1 = nullptr, *a2 = nullptr, *a3 = nullptr;  // BF16 [rows][32]
    float *logits = nullptr;                               // [rows]
    float *g = nullptr;                                    // dL/dlogits [rows]
    float *dz1 = nullptr, *dz2 = nullptr, *dz3 = nullptr;  // FP32 [rows][32]
    float *inv_valid = nullptr;
    int64_t *tiles_before = nullptr;                       // [S]
};

int64_t cnn_tiles(const std::vector<SeriesDesc> &desc, std::vector<int64_t> &tiles_before);
cudaError_t cnn_prepare(const CnnState &W, cudaStream_t st);
// Forward pass; wait_limit_ns bounds the tensor-core kernels' waits, whose expiry sets the
// timeout bit of *status (when not null).
cudaError_t cnn_forward(const CnnState &W, const uint16_t *feat, const CnnActs &A, const SeriesDesc *desc,
                        const int64_t *tiles_before, int64_t S, int64_t ntiles, long long wait_limit_ns,
                        int32_t *status, cudaStream_t st, const unsigned long long *gate = nullptr);
// One hidden layer (0: 18 -> 32, 1 and 2: 32 -> 32, ReLU, BF16 out) on the tcgen05 tensor cores.
cudaError_t cnn_hidden_tc(int layer, const __nv_bfloat16 *in, const float *W, const float *bias, __nv_bfloat16 *out,
                          const SeriesDesc *desc, const int64_t *tiles_before, int64_t S, int64_t ntiles,
                          long long wait_limit_ns, int32_t *status, cudaStream_t st,
                          const unsigned long long *gate = nullptr);
// Inference in one kernel (conv_tc.cu): logits of every step of every series, written at the
// feature rows of the steps (pad rows untouched).  Tiles of 116 positions; tiles_before is the
// prefix of cnn_infer_tiles.
int64_t cnn_infer_tiles(const std::vector<SeriesDesc> &desc, std::vector<int64_t> &tiles_before);
cudaError_t cnn_infer(const CnnState &W, const uint16_t *feat, float *logits, const SeriesDesc *desc,
                      const int64_t *tiles_before, int64_t S, int64_t ntiles, long long wait_limit_ns, int32_t *status,
                      cudaStream_t st, const unsigned long long *gate = nullptr);
cudaError_t cnn_backward(const CnnState &W, const uint16_t *feat, const CnnActs &A, const int32_t *cp_count,
                         const int32_t *cp_idx, int32_t max_cp, const SeriesDesc *desc, int64_t S, int T,
                         float *grad, float *loss, cudaStream_t st);
cudaError_t cnn_adam(CnnState &W, const float *grad, float lr, cudaStream_t st);
cudaError_t launch_zero_pad_rows(void *buf, int row_bytes, const SeriesDesc *desc, int64_t S, cudaStream_t st);
cudaError_t launch_propose(const float *logits, const SeriesDesc *desc, int64_t S, int32_t n_win, int32_t half,
                           int32_t *win_center, float *conf, cudaStream_t st, const unsigned long long *gate = nullptr);

}  // namespace mt4g
