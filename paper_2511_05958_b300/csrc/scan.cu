// All-splits KS scan, Kolmogorov p-value and binary segmentation, driven by a
// device work queue consumed by a persistent kernel.
//
// Scan (paper Sec. IV-B-1 (4): every index is a candidate; Sec. II-C-1: D =
// max_x |F(x) - G(x)|).  For a segment [lo, hi) of H steps and a split k
// (a = k - lo), with c_L(x), C(x) the left and pooled counts of samples <= x,
//     D_k = max_x |N c_L - n_L C| / (n_L n_R) = m g_k / (m^2 a (H - a)),
//     g_k = max_x |H c_L(x) - a C(x)|,
// because N = m H and n_L = m a.  |H c_L - a C| <= m a (H - a) <= m H^2 / 4, so
// when m H^2 < 2^33 the difference is exact in wrapping 32-bit arithmetic; larger
// shapes take the 64-bit path.
//
// Each thread of a 512-thread CTA owns one split k.  The CTA walks the series'
// runs of equal values (the run table built by the sort) in value order, so x
// takes every distinct value of the series; values absent from the segment leave
// the counts unchanged and cannot raise the maximum.  Within a run the labels are
// sorted, so the in-segment part is [lower_bound(lo), lower_bound(hi)) and the
// part left of k is one more lower_bound.  A warp fetches 32 runs' bounds at once
// (lane j owns run j0 + j) and broadcasts them with shuffles.
//
// p-value: lambda = num / sqrt(N den); Q(lambda) from the two standard series of the
// Kolmogorov survival function (the distribution behind Eq. 1), switched at 1.18,
// summed until a term < 1e-17 of the sum or 100 terms; lambda^2 > 345 -> 0.  All
// products and sums are explicit round-to-nearest operations so the result is the
// same IEEE sequence a plain C evaluation performs.
//
// Work queue: an item is (series, lo, hi, chunk); a segment with more than 512
// splits is split into chunks.  A CTA takes a ticket, waits (bounded, on the
// global timer) until that slot is published or no work is pending, scans, and the
// last chunk of a segment to finish combines the chunks' results, computes p and,
// if p <= alpha, records the change point and publishes the two children.
#include <climits>

#include "mt4g_internal.cuh"

namespace mt4g {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ long long ld_acquire_s64(const long long *p) {
    long long v;
    asm volatile("ld.acquire.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int lower_bound_lab(const uint16_t *__restrict__ lab, int a, int b, int v) {
    while (a < b) {
        const int mid = (a + b) >> 1;
        if ((int)__ldg(lab + mid) < v)
            a = mid + 1;
        else
            b = mid;
    }
    return a;
}

// ---------------------------------------------------------------- p-value

__device__ double kolmogorov_q(double lam) {
    const double PI2 = 9.8696044010893586188;
    const double SQRT_2PI = 2.5066282746310005024;
    if (!(lam > 0.0)) return 1.0;
    const double l2 = __dmul_rn(lam, lam);
    if (l2 > 345.0) return 0.0;
    double q;
    if (lam < 1.18) {
        double s = 0.0;
        const double den = __dmul_rn(8.0, l2);
        for (int j = 1; j <= 100; j++) {
            const double o = (double)(2 * j - 1);
            const double e = __ddiv_rn(__dmul_rn(-__dmul_rn(o, o), PI2), den);
            const double term = exp(e);
            s = __dadd_rn(s, term);
            if (term < __dmul_rn(1e-17, s)) break;
        }
        q = __dsub_rn(1.0, __dmul_rn(__ddiv_rn(SQRT_2PI, lam), s));
    } else {
        double s = 0.0;
        for (int j = 1; j <= 100; j++) {
            const double jj = (double)j;
            const double term = exp(__dmul_rn(__dmul_rn(__dmul_rn(-2.0, jj), jj), l2));
            s = (j & 1) ? __dadd_rn(s, term) : __dsub_rn(s, term);
            if (term < __dmul_rn(1e-17, fabs(s))) break;
        }
        q = __dmul_rn(2.0, s);
    }
    if (q < 0.0) q = 0.0;
    if (q > 1.0) q = 1.0;
    return q;
}

__device__ double ks_pvalue(int64_t num, int64_t den, int64_t N) {
    if (num <= 0) return 1.0;
    const double lam = __ddiv_rn((double)num, __dsqrt_rn(__dmul_rn((double)N, (double)den)));
    return kolmogorov_q(lam);
}

// ---------------------------------------------------------------- comparisons

constexpr int kNoK = INT_MAX;

// D(k1) > D(k2), or equal D and k1 < k2, with D(k) = g / (a (H - a)).
__device__ __forceinline__ bool better(int k1, uint64_t g1, int k2, uint64_t g2, int lo, int hi) {
    if (k2 == kNoK) return k1 != kNoK;
    if (k1 == kNoK) return false;
    const uint64_t d1 = (uint64_t)(k1 - lo) * (uint64_t)(hi - k1);
    const uint64_t d2 = (uint64_t)(k2 - lo) * (uint64_t)(hi - k2);
    const uint64_t lh = __umul64hi(g1, d2), ll = g1 * d2;
    const uint64_t rh = __umul64hi(g2, d1), rl = g2 * d1;
    if (lh != rh) return lh > rh;
    if (ll != rl) return ll > rl;
    return k1 < k2;
}

// ---------------------------------------------------------------- scan of one chunk

template <bool WIDE>
__device__ uint64_t scan_runs(const uint16_t *__restrict__ lab, const int32_t *__restrict__ rt, int U, int T,
                              int lo, int hi, int k, int &nonempty) {
    const int lane = threadIdx.x & 31;
    const uint32_t H = (uint32_t)(hi - lo);
    const uint32_t a = (uint32_t)(k - lo);
    uint32_t cl = 0, C = 0;
    uint64_t mx = 0;
    uint32_t mx32 = 0;
    nonempty = 0;
    for (int j0 = 0; j0 < U; j0 += 32) {
        const int j = j0 + lane;
        int si = 0, ei = 0, fi = 0, la = 0;
        if (j < U) {
            const int a0 = __ldg(rt + j), b0 = __ldg(rt + j + 1);
            si = (lo == 0) ? a0 : lower_bound_lab(lab, a0, b0, lo);
            ei = (hi == T) ? b0 : lower_bound_lab(lab, si, b0, hi);
            if (ei > si) {
                fi = __ldg(lab + si);
                la = __ldg(lab + ei - 1);
            }
        }
        const int nr = min(32, U - j0);
        for (int r = 0; r < nr; r++) {
            const int rsi = __shfl_sync(kFull, si, r);
            const int rei = __shfl_sync(kFull, ei, r);
            if (rsi == rei) continue;  // no sample of this value inside the segment
            nonempty++;
            const int rfi = __shfl_sync(kFull, fi, r);
            const int rla = __shfl_sync(kFull, la, r);
            const uint32_t cnt = (uint32_t)(rei - rsi);
            C += cnt;
            if (rla < k)
                cl += cnt;
            else if (rfi < k)
                cl += (uint32_t)(lower_bound_lab(lab, rsi, rei, k) - rsi);
            if (WIDE) {
                const int64_t f = (int64_t)H * cl - (int64_t)a * C;
                const uint64_t af = (uint64_t)(f < 0 ? -f : f);
                mx = af > mx ? af : mx;
            } else {
                const int32_t f = (int32_t)(H * cl - a * C);
                const uint32_t af = (uint32_t)(f < 0 ? -f : f);
                mx32 = max(mx32, af);
            }
        }
    }
    return WIDE ? mx : (uint64_t)mx32;
}

// ---------------------------------------------------------------- queue helpers

// Publish the chunks of the children of a split.  Called by one thread.
__device__ void push_children(const RunParams &P, int series, int lo, int k, int hi, uint32_t epoch) {
    const int cl_n = seg_chunks(k - lo, P.min_seg);
    const int cr_n = seg_chunks(hi - k, P.min_seg);
    const int tot = cl_n + cr_n;
    if (tot == 0) return;
    atomicAdd((unsigned long long *)&P.q->pending, (unsigned long long)tot);
    const unsigned long long base = atomicAdd(&P.q->tail, (unsigned long long)tot);
    if (base + tot > P.q->cap) {
        atomicOr(&P.q->status, kStatusQueueFull);
        atomicAdd((unsigned long long *)&P.q->pending, (unsigned long long)(-(long long)tot));
        return;
    }
    for (int c = 0; c < cl_n; c++) P.items[base + c] = WorkItem{series, lo, k, c};
    for (int c = 0; c < cr_n; c++) P.items[base + cl_n + c] = WorkItem{series, k, hi, c};
    __threadfence();
    for (int c = 0; c < tot; c++) st_release_u32((uint32_t *)P.ready + base + c, epoch);
}

__device__ void finish_segment(const RunParams &P, const SeriesDesc &d, int series, int lo, int hi, int k,
                               uint64_t g, uint32_t epoch) {
    const int64_t m = d.m;
    const int64_t a = k - lo, b = hi - k;
    const int64_t num = m * (int64_t)g;
    const int64_t den = (m * a) * (m * b);
    const int64_t N = m * (int64_t)(hi - lo);
    const double p = ks_pvalue(num, den, N);
    if (P.mode == kRunScan) {
        P.k_out[series] = k;
        P.dnum_out[series] = num;
        P.dden_out[series] = den;
        P.p_out[series] = p;
        return;
    }
    if (p <= P.alpha) {
        const int64_t slot = d.step_base + k;
        P.cp_num[slot] = num;
        P.cp_den[slot] = den;
        P.cp_p[slot] = p;
        P.cp_flag[slot] = 1;
        push_children(P, series, lo, k, hi, epoch);
    }
}

__global__ void __launch_bounds__(kScanThreads, 2) queue_kernel(RunParams P, uint32_t epoch) {
    __shared__ WorkItem s_item;
    __shared__ unsigned long long s_ticket;
    __shared__ int s_state;
    __shared__ int s_k[kScanThreads / 32];
    __shared__ uint64_t s_g[kScanThreads / 32];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned long long cap = P.q->cap;

    for (;;) {
        if (tid == 0) {
            const unsigned long long ticket = atomicAdd(&P.q->head, 1ull);
            const unsigned long long t0 = globaltimer_ns();
            unsigned ns = 32;
            int state = 0;
            for (;;) {
                if (ticket < cap && ld_acquire_u32((const uint32_t *)P.ready + ticket) >= epoch) {
                    const int4 raw = __ldcg((const int4 *)(P.items + ticket));
                    s_item = WorkItem{raw.x, raw.y, raw.z, raw.w};
                    state = 1;
                    break;
                }
                if (ld_acquire_s64(&P.q->pending) <= 0) break;
                if (globaltimer_ns() - t0 > (unsigned long long)P.wait_limit_ns) {
                    atomicOr(&P.q->status, kStatusTimeout);
                    break;
                }
                __nanosleep(ns);
                ns = ns < 1024 ? ns * 2 : 1024;
            }
            s_state = state;
            s_ticket = ticket;
        }
        __syncthreads();
        if (s_state == 0) return;
        const unsigned long long ticket = s_ticket;
        const WorkItem it = s_item;
        const SeriesDesc d = P.desc[it.series];
        const int lo = it.lo, hi = it.hi;
        const int kfirst = lo + P.min_seg + it.chunk * kChunkK;
        const int klast = min(kfirst + kChunkK - 1, hi - P.min_seg);
        const int k = kfirst + tid;
        const bool active = k <= klast;
        const int U = d.nruns;
        const int32_t *rt = P.runs + d.run_base;
        const uint16_t *lab = P.lab + d.off;
        const uint64_t H = (uint64_t)(hi - lo);
        const bool wide = (uint64_t)d.m * H * H >= (1ull << 33);
        int nonempty = 0;
        uint64_t g = wide ? scan_runs<true>(lab, rt, U, d.T, lo, hi, k, nonempty)
                          : scan_runs<false>(lab, rt, U, d.T, lo, hi, k, nonempty);

        // block argmax of D, ties to the smallest k
        int bk = active ? k : kNoK;
        uint64_t bg = active ? g : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int k2 = __shfl_down_sync(kFull, bk, o);
            const uint64_t g2 = __shfl_down_sync(kFull, bg, o);
            if (better(k2, g2, bk, bg, lo, hi)) {
                bk = k2;
                bg = g2;
            }
        }
        if (lane == 0) {
            s_k[warp] = bk;
            s_g[warp] = bg;
        }
        __syncthreads();
        if (tid == 0) {
            atomicAdd(&P.q->evals, (unsigned long long)(klast - kfirst + 1) * (unsigned long long)nonempty);
            for (int w = 1; w < kScanThreads / 32; w++)
                if (better(s_k[w], s_g[w], bk, bg, lo, hi)) {
                    bk = s_k[w];
                    bg = s_g[w];
                }
            const int nch = seg_chunks(hi - lo, P.min_seg);
            if (nch == 1) {
                finish_segment(P, d, it.series, lo, hi, bk, bg, epoch);
            } else {
                // write this chunk's result over its consumed slot; the last chunk combines
                ChunkResult cr{bk, 0, bg};
                *reinterpret_cast<ChunkResult *>(P.items + ticket) = cr;
                __threadfence();
                const unsigned long long base = ticket - (unsigned long long)it.chunk;
                const uint32_t old = atomicAdd((uint32_t *)P.ready + base, 1u);
                if (old == epoch + (uint32_t)nch - 1u) {
                    __threadfence();
                    int ck = kNoK;
                    uint64_t cg = 0;
                    for (int c = 0; c < nch; c++) {
                        const int4 raw = __ldcg((const int4 *)(P.items + base + c));
                        const int k2 = raw.x;
                        const uint64_t g2 = (uint64_t)(uint32_t)raw.z | ((uint64_t)(uint32_t)raw.w << 32);
                        if (better(k2, g2, ck, cg, lo, hi)) {
                            ck = k2;
                            cg = g2;
                        }
                    }
                    finish_segment(P, d, it.series, lo, hi, ck, cg, epoch);
                }
            }
            __threadfence();
            atomicAdd((unsigned long long *)&P.q->pending, (unsigned long long)(-1ll));
        }
        __syncthreads();
    }
}

// One warp per series: gather the flagged steps in ascending order.
__global__ void collect_kernel(const SeriesDesc *__restrict__ desc, int64_t S, const uint8_t *__restrict__ cp_flag,
                               const int64_t *__restrict__ cp_num, const int64_t *__restrict__ cp_den,
                               const double *__restrict__ cp_p, int32_t max_cp, int32_t *cp_count, int32_t *cp_idx,
                               int64_t *dnum, int64_t *dden, double *p, QueueHeader *q) {
    const int64_t s = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (s >= S) return;
    const SeriesDesc d = desc[s];
    int32_t count = 0;
    for (int t0 = 0; t0 < d.T; t0 += 32) {
        const int t = t0 + lane;
        const bool f = t < d.T && cp_flag[d.step_base + t];
        const unsigned b = __ballot_sync(kFull, f);
        if (f) {
            const int pos = count + __popc(b & ((1u << lane) - 1u));
            if (pos < max_cp) {
                const int64_t o = s * max_cp + pos;
                cp_idx[o] = t;
                dnum[o] = cp_num[d.step_base + t];
                dden[o] = cp_den[d.step_base + t];
                p[o] = cp_p[d.step_base + t];
            }
        }
        count += __popc(b);
    }
    for (int pos = count + lane; pos < max_cp; pos += 32) {
        const int64_t o = s * max_cp + pos;
        cp_idx[o] = -1;
        dnum[o] = 0;
        dden[o] = 0;
        p[o] = 1.0;
    }
    if (lane == 0) {
        cp_count[s] = count;
        if (count > max_cp) atomicOr(&q->status, kStatusCapacity);
    }
}

}  // namespace

int queue_grid(int device) {
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, queue_kernel, kScanThreads, 0) != cudaSuccess)
        return 0;
    return sms * (per_sm > 0 ? per_sm : 1);
}

cudaError_t launch_queue_run(const RunParams &P, int grid, uint32_t epoch, cudaStream_t st) {
    queue_kernel<<<grid, kScanThreads, 0, st>>>(P, epoch);
    return cudaGetLastError();
}

cudaError_t launch_collect(const SeriesDesc *desc, int64_t S, const uint8_t *cp_flag, const int64_t *cp_num,
                           const int64_t *cp_den, const double *cp_p, int32_t max_cp, int32_t *cp_count,
                           int32_t *cp_idx, int64_t *dnum, int64_t *dden, double *p, QueueHeader *q,
                           cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    const int warps = 8;
    const unsigned blocks = (unsigned)((S + warps - 1) / warps);
    collect_kernel<<<blocks, warps * 32, 0, st>>>(desc, S, cp_flag, cp_num, cp_den, cp_p, max_cp, cp_count, cp_idx,
                                                  dnum, dden, p, q);
    return cudaGetLastError();
}

}  // namespace mt4g
