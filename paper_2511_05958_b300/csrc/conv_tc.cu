// Hidden layers of the proposal network on the 5th-generation tensor cores (tcgen05).
//
// A width-5 convolution along the steps, out[p][o] = b[o] + sum_{d, i} x[p + d - 2][i] W[d][i][o],
// is a dense contraction: for a tile of 128 positions it is D[128 x 32] = sum over the five taps d
// of A_d[128 x 32] B_d[32 x 32]^T, with A_d the tile's input rows shifted by d and B_d[o][i] =
// W[d][i][o].  Each CTA keeps the five B_d in shared memory (BF16), builds the five shifted A_d of
// a tile in shared memory, and one thread issues ten tcgen05.mma (kind::f16, BF16 x BF16 -> FP32,
// M = 128, N = 32, K = 16) accumulating in tensor memory (32 columns); tcgen05.commit signals an
// mbarrier when they are done, every thread reads its position's 32 sums with tcgen05.ld, adds the
// bias, applies ReLU and stores BF16.  CTAs are persistent over the tiles.  Each of a tile's 132
// input rows is read from global memory once (16-byte chunks of 8 channels, at most five chunks per
// thread, held in registers) and written to the five shifted operands in shared memory; the next
// tile's chunks are loaded while the current tile's MMAs run.
//
// Shared-memory operands use the canonical K-major layout without swizzle: 8-row x 16-byte core
// matrices stored contiguously, consecutive in K 128 bytes apart (the descriptor's leading byte
// offset) and consecutive 8-row groups 512 bytes apart (stride byte offset, K = 32).  Input rows
// of the first layer (18 channels) are padded to 32 channels with zeros; so are its weights.
//
// The mbarrier wait is bounded by the global timer; on expiry the kernel sets the timeout bit
// of *status (when given) and returns without writing further tiles.
#include <cuda_bf16.h>

#include "mt4g_cnn.cuh"

namespace mt4g {

namespace {

constexpr int kTcTile = 128;          // positions per tile: the MMA's M
constexpr int kTcRows = kTcTile + 4;  // with the two halo rows on each side
constexpr int kTcThreads = 128;
constexpr int kStatusTimeoutBit = 1;  // kStatusTimeout of the queue header

struct TcSmem {
    uint8_t a[5][kTcTile * 32 * 2];  // A_d, K-major core matrices (8 KB each)
    uint8_t b[5][32 * 32 * 2];       // B_d = W_d^T, K-major (2 KB each)
    float bias[32];
    uint64_t mbar;
    uint32_t tmem;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) in a K-major tile of K = 32 columns
__device__ __forceinline__ uint32_t kmaj32(int r, int k) { return ((r >> 3) * 4 + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2; }

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    constexpr uint64_t lbo = 128, sbo = 512;
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ int64_t tile_series(const int64_t *__restrict__ tiles_before, int64_t S, int64_t tile) {
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

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// 8 channels [8 kc, 8 kc + 8) of input row `row` (BF16), zero beyond CIN.
template <int CIN>
__device__ __forceinline__ uint4 load_chunk(const __nv_bfloat16 *__restrict__ in, int64_t row, int kc) {
    if constexpr (CIN == 32) {
        return __ldg(reinterpret_cast<const uint4 *>(in + row * 32) + kc);
    } else {
        // rows of CIN (even) BF16 values are 4-byte aligned: channel pairs as 32-bit words
        const uint32_t *src = reinterpret_cast<const uint32_t *>(in + row * CIN);
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int c = kc * 8 + 2 * j;
            w[j] = c < CIN ? __ldg(src + c / 2) : 0u;
        }
        return make_uint4(w[0], w[1], w[2], w[3]);
    }
}

template <int CIN>
__global__ void __launch_bounds__(kTcThreads) conv_tc_kernel(const __nv_bfloat16 *__restrict__ in,
                                                             const float *__restrict__ W,
                                                             const float *__restrict__ bias,
                                                             __nv_bfloat16 *__restrict__ out,
                                                             const SeriesDesc *__restrict__ desc,
                                                             const int64_t *__restrict__ tiles_before, int64_t S,
                                                             int64_t ntiles, long long wait_limit_ns,
                                                             int32_t *status,
                                                             const unsigned long long *__restrict__ gate) {
    if (gate && *gate == 0ull) return;  // before any barrier or tensor-memory allocation
    extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
    TcSmem &sm = *reinterpret_cast<TcSmem *>(tc_smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5;

    // B_d[o][i] = W[d][i][o] (BF16-rounded already), zero for the padded input channels
    for (int e = tid; e < 5 * 32 * 32; e += kTcThreads) {
        const int d = e >> 10, o = (e >> 5) & 31, i = e & 31;
        const float v = i < CIN ? W[(d * CIN + i) * 32 + o] : 0.f;
        *reinterpret_cast<__nv_bfloat16 *>(sm.b[d] + kmaj32(o, i)) = __float2bfloat16_rn(v);
    }
    if (tid < 32) sm.bias[tid] = bias[tid];
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(&sm.tmem)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = sm.tmem;
    // instruction descriptor: F32 accumulator, BF16 A and B, both K-major, N = 32, M = 128
    constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
    uint32_t phase = 0;

    // a tile's input rows as 16-byte chunks: chunk e = 4 row + kc, rows 0 .. kTcRows - 1 from the
    // tile's window start, thread tid holding e = tid + 128 j (j < kChunks), zero past the series
    constexpr int kChunks = (kTcRows * 4 + kTcThreads - 1) / kTcThreads;
    uint4 cur[kChunks];
    auto load_tile = [&](int64_t tile, uint4 (&dst)[kChunks]) {
        const int64_t s = tile_series(tiles_before, S, tile);
        const SeriesDesc d = desc[s];
        const int t0 = (int)(tile - tiles_before[s]) * kTcTile;
        const int64_t r0 = row_base(d, s) + t0;
        const int nrows = min(kTcRows, d.T + 4 - t0);
#pragma unroll
        for (int j = 0; j < kChunks; j++) {
            const int e = tid + kTcThreads * j, row = e >> 2, kc = e & 3;
            dst[j] = (row < nrows) ? load_chunk<CIN>(in, r0 + row, kc) : make_uint4(0, 0, 0, 0);
        }
    };
    if (blockIdx.x < ntiles) load_tile(blockIdx.x, cur);

    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t s = tile_series(tiles_before, S, tile);
        const SeriesDesc d = desc[s];
        const int t0 = (int)(tile - tiles_before[s]) * kTcTile;
        const int64_t r0 = row_base(d, s) + t0;  // padded row of the window start of position t0
        // the five shifted copies A_dd[r] = row r + dd of the tile: each chunk goes to every
        // (dd, r = row - dd) with 0 <= r < 128
#pragma unroll
        for (int j = 0; j < kChunks; j++) {
            const int e = tid + kTcThreads * j, row = e >> 2, kc = e & 3;
            if (row < kTcRows) {
#pragma unroll
                for (int dd = 0; dd < 5; dd++) {
                    const int r = row - dd;
                    if (r >= 0 && r < kTcTile) *reinterpret_cast<uint4 *>(sm.a[dd] + kmaj32(r, kc * 8)) = cur[j];
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
#pragma unroll
            for (int dd = 0; dd < 5; dd++)
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const uint64_t da = smem_desc(smem_u32(sm.a[dd]) + h * 256);
                    const uint64_t db = smem_desc(smem_u32(sm.b[dd]) + h * 256);
                    const uint32_t acc = (dd | h) ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(da), "l"(db), "r"(idesc), "r"(acc));
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&sm.mbar)));
        }
        // the next tile's chunks, in flight while the MMAs run
        if (tile + gridDim.x < ntiles) load_tile(tile + gridDim.x, cur);
        // bounded wait for the ten MMAs
        uint32_t done = 0;
        const unsigned long long w0 = globaltimer_ns();
        while (!done) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(smem_u32(&sm.mbar)), "r"(phase));
            if (!done && globaltimer_ns() - w0 > (unsigned long long)wait_limit_ns) break;
        }
        if (!__syncthreads_and((int)done)) {
            if (tid == 0 && status) atomicOr(status, kStatusTimeoutBit);
            break;
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        uint32_t acc[32];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
            "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(acc[0]), "=r"(acc[1]), "=r"(acc[2]), "=r"(acc[3]), "=r"(acc[4]), "=r"(acc[5]), "=r"(acc[6]),
              "=r"(acc[7]), "=r"(acc[8]), "=r"(acc[9]), "=r"(acc[10]), "=r"(acc[11]), "=r"(acc[12]), "=r"(acc[13]),
              "=r"(acc[14]), "=r"(acc[15]), "=r"(acc[16]), "=r"(acc[17]), "=r"(acc[18]), "=r"(acc[19]),
              "=r"(acc[20]), "=r"(acc[21]), "=r"(acc[22]), "=r"(acc[23]), "=r"(acc[24]), "=r"(acc[25]),
              "=r"(acc[26]), "=r"(acc[27]), "=r"(acc[28]), "=r"(acc[29]), "=r"(acc[30]), "=r"(acc[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (t0 + tid < d.T) {
            uint32_t packed[16];
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const float lo = fmaxf(__uint_as_float(acc[2 * j]) + sm.bias[2 * j], 0.f);
                const float hi = fmaxf(__uint_as_float(acc[2 * j + 1]) + sm.bias[2 * j + 1], 0.f);
                const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
                packed[j] = *reinterpret_cast<const uint32_t *>(&v);
            }
            uint4 *dst = reinterpret_cast<uint4 *>(out + (r0 + 2 + tid) * 32);
#pragma unroll
            for (int q = 0; q < 4; q++)
                dst[q] = make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
        }
        // every thread has read the accumulator before the next tile's MMAs overwrite it
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
}

template <int CIN>
cudaError_t launch_one(const __nv_bfloat16 *in, const float *W, const float *bias, __nv_bfloat16 *out,
                       const SeriesDesc *desc, const int64_t *tiles_before, int64_t S, int64_t ntiles,
                       long long wait_limit_ns, int32_t *status, cudaStream_t st,
                       const unsigned long long *gate) {
    static int configured_device = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_device != dev) {
        e = cudaFuncSetAttribute(conv_tc_kernel<CIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TcSmem));
        if (e != cudaSuccess) return e;
        configured_device = dev;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)sms * 4);
    conv_tc_kernel<CIN><<<(unsigned)grid, kTcThreads, sizeof(TcSmem), st>>>(in, W, bias, out, desc, tiles_before, S,
                                                                             ntiles, wait_limit_ns, status, gate);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Inference: the whole network in one kernel.  A tile is a window of kFzRows = 132 consecutive
// positions P .. P + 131 of one series; the three hidden layers run on 128-row MMAs (M = 128) and
// each loses two rows of context on either side, so layer L holds positions P + 2L .. P + 2L + 127
// and the last layer (32 -> 1, on CUDA cores) gives the kFzOut = 116 logits of positions
// P + 8 .. P + 123; consecutive tiles of a series start 116 positions apart (P = -8, 108, ...).
// Activations stay in shared memory; rows at positions outside [0, T) are zero at every layer,
// which is the zero padding of each convolution.  Four CTAs of 48 KB share an SM, each with one
// tile in flight; the next tile's input is copied while layers 2 and 3 run.
//
// Operand layout: each buffer stores, for every 8-channel chunk kc, a column of rows 16 bytes
// apart (row r of chunk kc at kc * kFzLbo + 16 r).  This is the K-major no-swizzle canonical
// layout with 8-row core matrices 128 bytes apart along M and chunks kFzLbo bytes apart along K,
// so the operand of tap d (rows d .. d + 127) is the same buffer with its start 16 d bytes later:
// one copy of the input serves all five taps.  The hidden layers' sums and their ReLU/BF16
// rounding are those of conv_tc_kernel (same MMAs in the same order); the last layer sums its
// products in four partial sums (one per 8-channel chunk), so its rounding differs from the
// layer-by-layer path's single chain.
constexpr int kFzRows = kTcRows;             // 132 rows per operand buffer
constexpr int kFzOut = kTcTile - 12;         // 116 logits per tile
constexpr int kFzLbo = kFzRows * 16;         // bytes between the chunks of a buffer
constexpr int kFzBLbo = 32 * 16;             // the same for the 32-row weight operands

struct FzSmem {
    uint8_t x[4 * kFzLbo];          // input window (the next tile's is copied once layer 1 is done)
    uint8_t h[4 * kFzLbo];          // hidden activations: each layer's epilogue overwrites its
                                    // own input once the layer's MMAs have completed
    uint8_t b[3][5][4 * kFzBLbo];   // B_d of the three hidden layers, B_d[o][i] = W[d][i][o]
    float bias[3][32];
    float w4[5 * 32];
    float b4;
    uint64_t mbar;
    uint32_t tmem;
};

__device__ __forceinline__ uint64_t col_desc(uint32_t addr, uint32_t lbo) {
    constexpr uint64_t sbo = 128;
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((sbo >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void fz_cp_async4(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}

__global__ void __launch_bounds__(kTcThreads, 4) cnn_infer_kernel(const uint32_t *__restrict__ feat,
                                                                  const float *__restrict__ Wu,
                                                                  float *__restrict__ logits,
                                                                  const SeriesDesc *__restrict__ desc,
                                                                  const int64_t *__restrict__ tiles_before, int64_t S,
                                                                  int64_t ntiles, long long wait_limit_ns,
                                                                  int32_t *status,
                                                                  const unsigned long long *__restrict__ gate) {
    if (gate && *gate == 0ull) return;  // before any barrier or tensor-memory allocation
    extern __shared__ __align__(1024) uint8_t fz_smem_raw[];
    FzSmem &sm = *reinterpret_cast<FzSmem *>(fz_smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    // this CTA's tiles: a contiguous range, so the series of the next tile is the same or a later one
    const int64_t tbeg = ntiles * blockIdx.x / gridDim.x, tend = ntiles * (blockIdx.x + 1) / gridDim.x;

    // weights: B_d of the hidden layers (first layer's 18 input channels padded to 32 with zeros)
#pragma unroll 4
    for (int e = tid; e < 3 * 5 * 32 * 32; e += kTcThreads) {
        const int L = e / 5120, d = (e >> 10) % 5, o = (e >> 5) & 31, i = e & 31;
        float v;
        if (L == 0)
            v = i < kFeatC ? Wu[cnn_off(0) + (d * kFeatC + i) * 32 + o] : 0.f;
        else
            v = Wu[cnn_off(2 * L) + (d * 32 + i) * 32 + o];
        *reinterpret_cast<__nv_bfloat16 *>(sm.b[L][d] + (i >> 3) * kFzBLbo + o * 16 + (i & 7) * 2) =
            __float2bfloat16_rn(v);
    }
    for (int e = tid; e < 3 * 32; e += kTcThreads) sm.bias[e / 32][e % 32] = Wu[cnn_off(1 + 2 * (e / 32)) + e % 32];
    for (int e = tid; e < 160; e += kTcThreads) sm.w4[e] = Wu[cnn_off(6) + e];
    if (tid == 0) sm.b4 = Wu[cnn_off(7)];
    // never written by the tiles: input channels 18 .. 31 and hidden rows 128 .. 131
    for (int e = tid; e < kFzRows * 7; e += kTcThreads) {
        const int r = e / 7, w = 9 + e % 7;
        *reinterpret_cast<uint32_t *>(sm.x + (w >> 2) * kFzLbo + r * 16 + (w & 3) * 4) = 0u;
    }
    if (tid < 16)
        *reinterpret_cast<uint4 *>(sm.h + (tid >> 2) * kFzLbo + (kTcTile + (tid & 3)) * 16) = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(&sm.tmem)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = sm.tmem;
    constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
    uint32_t phase = 0;

    // series of a tile, walking forward from the previous one
    int64_t s = 0;
    if (tbeg < tend) s = tile_series(tiles_before, S, tbeg);
    auto series_of = [&](int64_t tile) {
        while (s + 1 < S && tiles_before[s + 1] <= tile) s++;
        return s;
    };
    // copy tile `tile`'s input window into x: feature words (two channels each) 0 .. 8 of the
    // rows at positions P .. P + 131, zeros at positions outside [0, T)
    auto issue_x = [&](int64_t tile) {
        const int64_t ss = series_of(tile);
        const SeriesDesc d = desc[ss];
        const int P = (int)(tile - tiles_before[ss]) * kFzOut - 8;
        const uint32_t *src = feat + (row_base(d, ss) + 2) * (kFeatC / 2);  // position 0
        const uint32_t xa = smem_u32(sm.x);
        for (int e = tid; e < kFzRows * 9; e += kTcThreads) {
            const int j = e / 9, w = e - 9 * j, pos = P + j;
            const uint32_t dst = xa + (uint32_t)((w >> 2) * kFzLbo + j * 16 + (w & 3) * 4);
            if (pos >= 0 && pos < d.T)
                fz_cp_async4(dst, src + (int64_t)pos * (kFeatC / 2) + w);
            else
                asm volatile("st.shared.u32 [%0], %1;" ::"r"(dst), "r"(0u) : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // ten MMAs of one hidden layer: A = rows d .. d + 127 of buffer a, B = layer L's B_d
    auto issue_layer = [&](const uint8_t *a, int L) {
#pragma unroll
        for (int dd = 0; dd < 5; dd++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const uint64_t da = col_desc(smem_u32(a) + h * 2 * kFzLbo + dd * 16, kFzLbo);
                const uint64_t db = col_desc(smem_u32(sm.b[L][dd]) + h * 2 * kFzBLbo, kFzBLbo);
                const uint32_t acc = (dd | h) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(acc));
            }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&sm.mbar)));
    };
    // bounded wait for the layer's MMAs; false (on every thread) when the limit ran out
    auto wait_layer = [&]() {
        uint32_t done = 0;
        const unsigned long long w0 = globaltimer_ns();
        while (!done) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(smem_u32(&sm.mbar)), "r"(phase));
            if (!done && globaltimer_ns() - w0 > (unsigned long long)wait_limit_ns) break;
        }
        if (!__syncthreads_and((int)done)) {
            if (tid == 0 && status) atomicOr(status, kStatusTimeoutBit);
            return false;
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        return true;
    };
    // this thread's row of the accumulator -> ReLU(sum + bias) in BF16, zero outside [0, T)
    auto epilogue = [&](uint8_t *out, int L, bool inside) {
        uint32_t acc[32];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
            "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(acc[0]), "=r"(acc[1]), "=r"(acc[2]), "=r"(acc[3]), "=r"(acc[4]), "=r"(acc[5]), "=r"(acc[6]),
              "=r"(acc[7]), "=r"(acc[8]), "=r"(acc[9]), "=r"(acc[10]), "=r"(acc[11]), "=r"(acc[12]), "=r"(acc[13]),
              "=r"(acc[14]), "=r"(acc[15]), "=r"(acc[16]), "=r"(acc[17]), "=r"(acc[18]), "=r"(acc[19]),
              "=r"(acc[20]), "=r"(acc[21]), "=r"(acc[22]), "=r"(acc[23]), "=r"(acc[24]), "=r"(acc[25]),
              "=r"(acc[26]), "=r"(acc[27]), "=r"(acc[28]), "=r"(acc[29]), "=r"(acc[30]), "=r"(acc[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        uint32_t packed[16];
#pragma unroll
        for (int j = 0; j < 16; j++) {
            const float lo = fmaxf(__uint_as_float(acc[2 * j]) + sm.bias[L][2 * j], 0.f);
            const float hi = fmaxf(__uint_as_float(acc[2 * j + 1]) + sm.bias[L][2 * j + 1], 0.f);
            const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
            packed[j] = inside ? *reinterpret_cast<const uint32_t *>(&v) : 0u;
        }
#pragma unroll
        for (int q = 0; q < 4; q++)
            *reinterpret_cast<uint4 *>(out + q * kFzLbo + tid * 16) =
                make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
    };

    if (tbeg < tend) issue_x(tbeg);
    bool ok = true;
    for (int64_t tile = tbeg; tile < tend && ok; tile++) {
        const int64_t ss = series_of(tile);
        const SeriesDesc d = desc[ss];
        const int P = (int)(tile - tiles_before[ss]) * kFzOut - 8;
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) issue_layer(sm.x, 0);
        // hidden layers: layer L's row tid is position P + 2 (L + 1) + tid
#pragma unroll 1
        for (int L = 0; L < 3 && ok; L++) {
            ok = wait_layer();
            if (!ok) break;
            if (L == 0 && tile + 1 < tend) issue_x(tile + 1);  // x is free: in flight for the rest
            const int pos = P + 2 * (L + 1) + tid;
            epilogue(sm.h, L, pos >= 0 && pos < d.T);
            if (L < 2 && tid == 0) issue_layer(sm.h, L + 1);
        }
        if (!ok) break;
        // last layer, 32 -> 1, from the third layer's rows tid .. tid + 4; one partial sum per
        // 8-channel chunk
        const int pos = P + 8 + tid;
        if (tid < kFzOut && pos < d.T) {
            float part[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int dd = 0; dd < 5; dd++) {
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const uint4 v = *reinterpret_cast<const uint4 *>(sm.h + c * kFzLbo + (tid + dd) * 16);
                    const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int hh = 0; hh < 4; hh++) {
                        const float lo = __uint_as_float(u[hh] << 16), hi = __uint_as_float(u[hh] & 0xffff0000u);
                        part[c] = fmaf(lo, sm.w4[dd * 32 + c * 8 + 2 * hh], part[c]);
                        part[c] = fmaf(hi, sm.w4[dd * 32 + c * 8 + 2 * hh + 1], part[c]);
                    }
                }
            }
            logits[row_base(d, ss) + 2 + pos] = sm.b4 + ((part[0] + part[1]) + (part[2] + part[3]));
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
}

}  // namespace

int64_t cnn_infer_tiles(const std::vector<SeriesDesc> &desc, std::vector<int64_t> &tiles_before) {
    tiles_before.resize(desc.size());
    int64_t n = 0;
    for (size_t s = 0; s < desc.size(); s++) {
        tiles_before[s] = n;
        n += (desc[s].T + kFzOut - 1) / kFzOut;
    }
    return n;
}

cudaError_t cnn_infer(const CnnState &W, const uint16_t *feat, float *logits, const SeriesDesc *desc,
                      const int64_t *tiles_before, int64_t S, int64_t ntiles, long long wait_limit_ns, int32_t *status,
                      cudaStream_t st, const unsigned long long *gate) {
    if (ntiles <= 0) return cudaSuccess;
    static int configured_device = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_device != dev) {
        e = cudaFuncSetAttribute(cnn_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FzSmem));
        if (e != cudaSuccess) return e;
        configured_device = dev;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)sms * 4);
    cnn_infer_kernel<<<(unsigned)grid, kTcThreads, sizeof(FzSmem), st>>>(
        reinterpret_cast<const uint32_t *>(feat), W.used, logits, desc, tiles_before, S, ntiles, wait_limit_ns,
        status, gate);
    return cudaGetLastError();
}

cudaError_t cnn_hidden_tc(int layer, const __nv_bfloat16 *in, const float *W, const float *bias, __nv_bfloat16 *out,
                          const SeriesDesc *desc, const int64_t *tiles_before, int64_t S, int64_t ntiles,
                          long long wait_limit_ns, int32_t *status, cudaStream_t st,
                          const unsigned long long *gate) {
    if (ntiles <= 0) return cudaSuccess;
    if (layer == 0)
        return launch_one<kFeatC>(in, W, bias, out, desc, tiles_before, S, ntiles, wait_limit_ns, status, st, gate);
    return launch_one<32>(in, W, bias, out, desc, tiles_before, S, ntiles, wait_limit_ns, status, st, gate);
}

}  // namespace mt4g
