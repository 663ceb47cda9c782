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
// Each lane of a warp owns one split k.  The warp walks the series' runs of equal
// values (the run table built by the sort) in value order, so x takes every distinct
// value of the series; values absent from the segment leave the counts unchanged and
// cannot raise the maximum.  Within a run the labels are sorted, so the in-segment
// part is [lower_bound(lo), lower_bound(hi)) and the part left of k is one more
// lower_bound.
//
// p-value: lambda = num / sqrt(N den); Q(lambda) from the two standard series of the
// Kolmogorov survival function (the distribution behind Eq. 1), switched at 1.18,
// summed until a term < 1e-17 of the sum or 100 terms; lambda^2 > 345 -> 0.  All
// products and sums are explicit round-to-nearest operations so the result is the
// same IEEE sequence a plain C evaluation performs.
//
// Work queue: an item is (series, lo, hi, chunk), the 32 splits of one slice of a
// segment, scanned by one warp.  A warp takes a ticket, waits (bounded, on the global
// timer) until that slot is published or no work is pending, scans, and the last slice
// of a segment to finish combines the slices' results, computes p and, if p <= alpha,
// records the change point and publishes the slices of the two children.
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

// ---------------------------------------------------------------- scan of one slice

constexpr int kShflMax = 8;  // differentiating samples counted by broadcast; more -> search

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

// Per-warp staging area: KPT + 1 boundary counts plus the run bounds, for 32 runs.
template <int KPT>
struct SliceStage {
    int si[32];
    int ei[32];
    int cb[KPT + 1][32];
};

union StageUnion {
    SliceStage<1> s1;
    SliceStage<2> s2;
    SliceStage<4> s4;
};

// Lower bound of v among the in-segment labels [si, ei) of a run whose first and last
// in-segment labels are fi and la, starting the search at `from`.
__device__ __forceinline__ int count_below(const uint16_t *__restrict__ lab, int si, int ei, int fi, int la,
                                           int from, int v) {
    if (v <= fi) return si;
    if (v > la) return ei;
    return lower_bound_lab(lab, from, ei, v);
}

// g_k = max over distinct values x of |H c_L(x) - a C(x)| for the KPT * 32 splits
// k = k0 + 32 q + lane (q < KPT) of one warp.
//
// The warp stages 32 runs at a time (lane = run): the in-segment part [si, ei) of the
// run (no search when the run's full label range lies inside or outside [lo, hi)), and
// cb[q] = its samples with label < k0 + 32 q, q = 0..KPT.  Samples below k0 + 32 q count
// for every lane of group q; only the cb[q+1] - cb[q] samples with labels in
// [k0 + 32 q, k0 + 32 q + 32) distinguish the lanes, and each lane counts those below its
// own k, by broadcast for up to kShflMax of them, else by a search in that short sorted
// slice.  Empty runs are compacted away; the walk visits the runs in value order.
template <bool WIDE, int KPT>
__device__ void scan_slice(const uint16_t *__restrict__ lab, const int32_t *__restrict__ rt, int U, int T, int lo,
                           int hi, int k0, SliceStage<KPT> &st, uint64_t (&g)[KPT], int &nonempty) {
    const int lane = threadIdx.x & 31;
    const uint32_t H = (uint32_t)(hi - lo);
    uint32_t cl[KPT], a[KPT], mx32[KPT];
    uint64_t mx[KPT];
    int kq[KPT];
#pragma unroll
    for (int q = 0; q < KPT; q++) {
        kq[q] = k0 + 32 * q + lane;
        a[q] = (uint32_t)(kq[q] - lo);
        cl[q] = 0;
        mx[q] = 0;
        mx32[q] = 0;
    }
    uint32_t C = 0;
    nonempty = 0;
    for (int j0 = 0; j0 < U; j0 += 32) {
        const int j = j0 + lane;
        int si = 0, ei = 0;
        int cb[KPT + 1];
#pragma unroll
        for (int q = 0; q <= KPT; q++) cb[q] = 0;
        if (j < U) {
            const int a0 = __ldg(rt + j), b0 = __ldg(rt + j + 1);
            const int f0 = __ldg(lab + a0), l0 = __ldg(lab + b0 - 1);
            si = (f0 >= lo) ? a0 : (l0 < lo ? b0 : lower_bound_lab(lab, a0, b0, lo));
            ei = (l0 < hi) ? b0 : (f0 >= hi ? a0 : lower_bound_lab(lab, si, b0, hi));
            if (ei > si) {
                const int fi = (si == a0) ? f0 : __ldg(lab + si);
                const int la = (ei == b0) ? l0 : __ldg(lab + ei - 1);
                int from = si;
#pragma unroll
                for (int q = 0; q <= KPT; q++) {
                    from = count_below(lab, si, ei, fi, la, from, k0 + 32 * q);
                    cb[q] = from - si;
                }
            }
        }
        const unsigned ne = __ballot_sync(kFull, ei > si);
        if (ei > si) {
            const int pos = __popc(ne & lanemask_lt());
            st.si[pos] = si;
            st.ei[pos] = ei;
#pragma unroll
            for (int q = 0; q <= KPT; q++) st.cb[q][pos] = cb[q];
        }
        __syncwarp();
        const int cnt = __popc(ne);
        for (int r = 0; r < cnt; r++) {
            const int rsi = st.si[r];
            C += (uint32_t)(st.ei[r] - rsi);
            int lo_c = st.cb[0][r];
#pragma unroll
            for (int q = 0; q < KPT; q++) {
                const int hi_c = st.cb[q + 1][r];
                uint32_t add = (uint32_t)lo_c;
                const int L = hi_c - lo_c;
                if (L > 0) {  // warp-uniform
                    const int sb = rsi + lo_c;
                    if (L <= kShflMax) {
                        const int mine = lane < L ? (int)__ldg(lab + sb + lane) : 0x7fffffff;
                        for (int t = 0; t < L; t++) add += (uint32_t)(__shfl_sync(kFull, mine, t) < kq[q]);
                    } else {
                        add += (uint32_t)(lower_bound_lab(lab, sb, sb + L, kq[q]) - sb);
                    }
                }
                cl[q] += add;
                lo_c = hi_c;
                if (WIDE) {
                    const int64_t f = (int64_t)H * cl[q] - (int64_t)a[q] * C;
                    const uint64_t af = (uint64_t)(f < 0 ? -f : f);
                    mx[q] = af > mx[q] ? af : mx[q];
                } else {
                    const int32_t f = (int32_t)(H * cl[q] - a[q] * C);
                    const uint32_t af = (uint32_t)(f < 0 ? -f : f);
                    mx32[q] = max(mx32[q], af);
                }
            }
        }
        nonempty += cnt;
        __syncwarp();
    }
#pragma unroll
    for (int q = 0; q < KPT; q++) g[q] = WIDE ? mx[q] : (uint64_t)mx32[q];
}

// ---------------------------------------------------------------- queue helpers

// Warp-wide argmax of D (ties to the smallest k); every lane ends with the result.
__device__ __forceinline__ void warp_best(int &bk, uint64_t &bg, int lo, int hi) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int k2 = __shfl_xor_sync(kFull, bk, o);
        const uint64_t g2 = __shfl_xor_sync(kFull, bg, o);
        if (better(k2, g2, bk, bg, lo, hi)) {
            bk = k2;
            bg = g2;
        }
    }
}

// Decide a finished segment (all lanes call with the same arguments): p-value, outputs,
// and if significant the change point and the children's slices.
__device__ void finish_segment(const RunParams &P, const SeriesDesc &d, int series, int lo, int hi, int k,
                               uint64_t g, uint32_t epoch) {
    const int lane = threadIdx.x & 31;
    int accept = 0;
    if (lane == 0) {
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
        } else if (p <= P.alpha) {
            const int64_t slot = d.step_base + k;
            P.cp_num[slot] = num;
            P.cp_den[slot] = den;
            P.cp_p[slot] = p;
            P.cp_flag[slot] = 1;
            accept = 1;
        }
    }
    accept = __shfl_sync(kFull, accept, 0);
    if (!accept) return;
    const int cl_n = seg_chunks(k - lo, P.min_seg, d.kpt);
    const int cr_n = seg_chunks(hi - k, P.min_seg, d.kpt);
    const int tot = cl_n + cr_n;
    if (tot == 0) return;
    unsigned long long base = 0;
    int ok = 0;
    if (lane == 0) {
        atomicAdd((unsigned long long *)&P.q->pending, (unsigned long long)tot);
        base = atomicAdd(&P.q->tail, (unsigned long long)tot);
        ok = base + tot <= P.q->cap;
        if (!ok) {
            atomicOr(&P.q->status, kStatusQueueFull);
            atomicAdd((unsigned long long *)&P.q->pending, (unsigned long long)(-(long long)tot));
        }
    }
    ok = __shfl_sync(kFull, ok, 0);
    base = __shfl_sync(kFull, base, 0);
    if (!ok) return;
    for (int c = lane; c < tot; c += 32)
        P.items[base + c] = c < cl_n ? WorkItem{series, lo, k, c} : WorkItem{series, k, hi, c - cl_n};
    __threadfence();
    for (int c = lane; c < tot; c += 32) st_release_u32((uint32_t *)P.ready + base + c, epoch);
}

// Persistent kernel: every warp independently takes tickets from the queue and scans
// one 32-split slice per ticket.  No block-level synchronisation.
// Scan one slice and reduce it to the warp's best (k, g); every lane gets the result.
template <bool WIDE, int KPT>
__device__ void slice_best(const RunParams &P, const SeriesDesc &d, int lo, int hi, int k0, int klast,
                           StageUnion &stage, int &bk, uint64_t &bg, int &nonempty) {
    const int lane = threadIdx.x & 31;
    uint64_t g[KPT];
    SliceStage<KPT> &st = *reinterpret_cast<SliceStage<KPT> *>(&stage);
    scan_slice<WIDE, KPT>(P.lab + d.off, P.runs + d.run_base, d.nruns, d.T, lo, hi, k0, st, g, nonempty);
    bk = kNoK;
    bg = 0;
#pragma unroll
    for (int q = 0; q < KPT; q++) {
        const int k = k0 + 32 * q + lane;
        if (k <= klast && better(k, g[q], bk, bg, lo, hi)) {
            bk = k;
            bg = g[q];
        }
    }
    warp_best(bk, bg, lo, hi);
}

// Persistent kernel: every warp independently takes tickets from the queue and scans
// one slice (32 * kpt splits of one segment) per ticket.  No block-level synchronisation.
__global__ void __launch_bounds__(kScanThreads, 4) queue_kernel(RunParams P, uint32_t epoch) {
    __shared__ StageUnion s_stage[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    StageUnion &stage = s_stage[warp];
    const unsigned long long cap = P.q->cap;
    unsigned long long my_evals = 0;

    for (;;) {
        unsigned long long ticket = 0;
        int4 raw = make_int4(0, 0, 0, 0);
        int state = 0;
        if (lane == 0) {
            ticket = atomicAdd(&P.q->head, 1ull);
            const unsigned long long t0 = globaltimer_ns();
            unsigned ns = 32;
            for (;;) {
                if (ticket < cap && ld_acquire_u32((const uint32_t *)P.ready + ticket) >= epoch) {
                    raw = __ldcg((const int4 *)(P.items + ticket));
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
        }
        state = __shfl_sync(kFull, state, 0);
        if (state == 0) break;
        ticket = __shfl_sync(kFull, ticket, 0);
        const WorkItem it{__shfl_sync(kFull, raw.x, 0), __shfl_sync(kFull, raw.y, 0), __shfl_sync(kFull, raw.z, 0),
                          __shfl_sync(kFull, raw.w, 0)};
        const SeriesDesc d = P.desc[it.series];
        const int lo = it.lo, hi = it.hi;
        const int kpt = d.kpt;
        const int k0 = lo + P.min_seg + it.chunk * 32 * kpt;
        const int klast = min(k0 + 32 * kpt - 1, hi - P.min_seg);
        const uint64_t H = (uint64_t)(hi - lo);
        const bool wide = (uint64_t)d.m * H * H >= (1ull << 33);
        int nonempty = 0, bk = kNoK;
        uint64_t bg = 0;
        if (kpt == 4) {
            if (wide) slice_best<true, 4>(P, d, lo, hi, k0, klast, stage, bk, bg, nonempty);
            else slice_best<false, 4>(P, d, lo, hi, k0, klast, stage, bk, bg, nonempty);
        } else if (kpt == 2) {
            if (wide) slice_best<true, 2>(P, d, lo, hi, k0, klast, stage, bk, bg, nonempty);
            else slice_best<false, 2>(P, d, lo, hi, k0, klast, stage, bk, bg, nonempty);
        } else {
            if (wide) slice_best<true, 1>(P, d, lo, hi, k0, klast, stage, bk, bg, nonempty);
            else slice_best<false, 1>(P, d, lo, hi, k0, klast, stage, bk, bg, nonempty);
        }
        my_evals += (unsigned long long)(klast - k0 + 1) * (unsigned long long)nonempty;

        const int nch = seg_chunks(hi - lo, P.min_seg, kpt);
        if (nch == 1) {
            finish_segment(P, d, it.series, lo, hi, bk, bg, epoch);
        } else {
            // write this slice's result over its consumed slot; the last slice combines
            const unsigned long long base = ticket - (unsigned long long)it.chunk;
            int last = 0;
            if (lane == 0) {
                *reinterpret_cast<ChunkResult *>(P.items + ticket) = ChunkResult{bk, 0, bg};
                __threadfence();
                const uint32_t old = atomicAdd((uint32_t *)P.ready + base, 1u);
                last = old == epoch + (uint32_t)nch - 1u;
            }
            last = __shfl_sync(kFull, last, 0);
            if (last) {
                __threadfence();
                int ck = kNoK;
                uint64_t cg = 0;
                for (int c = lane; c < nch; c += 32) {
                    const int4 r2 = __ldcg((const int4 *)(P.items + base + c));
                    const uint64_t g2 = (uint64_t)(uint32_t)r2.z | ((uint64_t)(uint32_t)r2.w << 32);
                    if (better(r2.x, g2, ck, cg, lo, hi)) {
                        ck = r2.x;
                        cg = g2;
                    }
                }
                warp_best(ck, cg, lo, hi);
                finish_segment(P, d, it.series, lo, hi, ck, cg, epoch);
            }
        }
        if (lane == 0) {
            __threadfence();
            atomicAdd((unsigned long long *)&P.q->pending, (unsigned long long)(-1ll));
        }
        __syncwarp();
    }
    if (lane == 0 && my_evals) atomicAdd(&P.q->evals, my_evals);
}

// Expand the top-level slices of every series into the queue, costliest series first.
__global__ void init_items_kernel(const SeriesDesc *__restrict__ desc, const int32_t *__restrict__ qorder,
                                  const int64_t *__restrict__ item_base, int64_t S, int32_t min_seg,
                                  WorkItem *items, int32_t *ready, uint32_t epoch) {
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= S) return;
    const int32_t s = qorder[i];
    const int32_t T = desc[s].T;
    const int nch = seg_chunks(T, min_seg, desc[s].kpt);
    const int64_t b = item_base[i];
    for (int c = lane; c < nch; c += 32) {
        items[b + c] = WorkItem{s, 0, T, c};
        ready[b + c] = (int32_t)epoch;
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

cudaError_t launch_init_items(const SeriesDesc *desc, const int32_t *qorder, const int64_t *item_base, int64_t S,
                              int32_t min_seg, WorkItem *items, int32_t *ready, uint32_t epoch, cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    const int warps = 8;
    init_items_kernel<<<(unsigned)((S + warps - 1) / warps), warps * 32, 0, st>>>(desc, qorder, item_base, S, min_seg,
                                                                                    items, ready, epoch);
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
