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
// Two ways to get g_k for every split.  Run sweep (series with at most kSweepMaxRuns
// distinct values, narrow shapes): one warp per segment walks the splits in order and moves
// one step's samples into the left part at a time (see sweep_best).  Slices (the rest): each
// lane of a warp owns one split k.  The warp walks the series' runs of equal
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
// Work queue: an item is one member of a group pushed together for a segment (the
// slices of a full scan, or a learned probe / refinement group), processed by one warp.
// A warp takes a ticket, waits (bounded, on the global timer) until that slot is
// published or no work is pending, processes it, writes its best split over its slot and
// counts itself done in the group's counter; the last member combines the group,
// computes p and, if p <= alpha, records the change point and pushes the children.
#include <algorithm>
#include <climits>
#include <type_traits>

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

// 128-bit test x1 * y1 < x2 * y2 for unsigned 64-bit operands.
__device__ __forceinline__ bool prod_less(uint64_t x1, uint64_t y1, uint64_t x2, uint64_t y2) {
    const uint64_t h1 = __umul64hi(x1, y1), l1 = x1 * y1;
    const uint64_t h2 = __umul64hi(x2, y2), l2 = x2 * y2;
    return h1 < h2 || (h1 == h2 && l1 < l2);
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

// Per-warp staging for one-group slices: (si, ei, cb0, cb1) of 32 runs as int4, and a
// 32-bin histogram for counting differentiating samples.
struct WarpStage {
    StageUnion u;
    int2 pre[32];   // inclusive prefix over the staged runs of (labels below k0, in-segment samples)
    int4 meta[32];  // per staged run with differentiating labels: (first such position, L | flags, M1, M2)
    uint4 lbl[32];  // up to 8 labels from that position (16-bit each), for runs with repeats
    int hist[32];
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
//
// One-group (32-split) slice, the common tile.  Staging (lane = run) also forms, over the
// batch, inclusive prefix sums of the labels below k0 and of the in-segment samples, so that
// at run r of the batch
//     H c_L - a C = K + H cbs_r - a ns_r,
// with K carried from the previous batches plus H times this lane's differentiating labels
// met so far.  A run without differentiating labels (most runs) then costs one shared load
// and the two multiply-adds, |.| and max of the definition.  For the others the lane's count
// comes from bit masks of the window offsets (first and second occurrences: two AND + POPC)
// when at most kShflMax labels fall in the window and none repeats more than twice, else from
// the staged labels, a 32-bin histogram, or a search.  The first kShflMax labels from the
// window start are loaded together during staging; they also give the window's end without a
// second search unless more than kShflMax labels fall in it.
template <bool WIDE>
__device__ void scan_slice1(const uint16_t *__restrict__ lab, const int32_t *__restrict__ rt, int U, int T, int lo,
                            int hi, int k0, WarpStage &ws, uint64_t &g_out, int &nonempty) {
    using Acc = typename std::conditional<WIDE, int64_t, uint32_t>::type;
    const int lane = threadIdx.x & 31;
    const int k = k0 + lane, k1 = k0 + 32;
    const unsigned lt = lanemask_lt();
    const Acc H = (Acc)(hi - lo);
    const Acc a = (Acc)(k - lo);
    // K = H c_L - a C over the runs walked so far (c_L counts labels below this lane's k); the
    // value at a run of the current batch is K + H (labels below k0 up to it) - a (samples up to it)
    // plus H times the lane's differentiating labels met so far.
    Acc K = 0;
    uint32_t mx32 = 0;
    uint64_t mx = 0;
    nonempty = 0;
    ws.hist[lane] = 0;
    __syncwarp();
    // the run bounds and end labels of the next batch are loaded one batch ahead: the run
    // bounds before this batch's staging, the end labels before its walk
    int na0 = 0, nb0 = 0, nf0 = 0, nl0 = 0;
    if (lane < U) {
        na0 = __ldg(rt + lane);
        nb0 = __ldg(rt + lane + 1);
        nf0 = __ldg(lab + na0);
        nl0 = __ldg(lab + nb0 - 1);
    }
    for (int j0 = 0; j0 < U; j0 += 32) {
        const int j = j0 + lane;
        int si = 0, ei = 0, c0 = 0, n_av = 0, L = 0;
        bool la_lt = false;
        const int a0 = na0, b0 = nb0, f0 = nf0, l0 = nl0;
        const int jn = j + 32;
        if (jn < U) {
            na0 = __ldg(rt + jn);
            nb0 = __ldg(rt + jn + 1);
        }
        if (j < U) {
            si = (f0 >= lo) ? a0 : (l0 < lo ? b0 : lower_bound_lab(lab, a0, b0, lo));
            ei = (l0 < hi) ? b0 : (f0 >= hi ? a0 : lower_bound_lab(lab, si, b0, hi));
            if (ei > si) {
                const int fi = (si == a0) ? f0 : __ldg(lab + si);
                const int la = (ei == b0) ? l0 : __ldg(lab + ei - 1);
                c0 = count_below(lab, si, ei, fi, la, si, k0);
                n_av = min(kShflMax, ei - c0);
                la_lt = la < k1;
            }
        }
        // The labels from c0 on are sorted: load up to kShflMax of them at once.  Those below k1
        // distinguish the lanes; the rest lie above every split of the slice.
        uint32_t pk[4] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu};
        uint32_t M1 = 0, M2 = 0;
        bool multi = false;
        int below = 0;
        if (n_av > 0) {
            const uint16_t *src = lab + c0;
#pragma unroll
            for (int q = 0; q < kShflMax; q++) {
                const uint32_t v = q < n_av ? (uint32_t)__ldg(src + q) : 0xffffu;
                pk[q >> 1] = (q & 1) ? ((pk[q >> 1] & 0xffffu) | (v << 16)) : ((pk[q >> 1] & 0xffff0000u) | v);
                if (v < (uint32_t)k1) {
                    // offsets from k0 as bits: first occurrences in M1, second in M2
                    const uint32_t bit = 1u << (v - (uint32_t)k0);
                    below++;
                    multi |= (M2 & bit) != 0;
                    M2 |= M1 & bit;
                    M1 |= bit;
                }
            }
        }
        if (ei > si) {
            if (la_lt)
                L = ei - c0;
            else if (below < n_av || n_av == ei - c0)
                L = below;
            else
                L = lower_bound_lab(lab, c0 + n_av, ei, k1) - c0;
        }
        // inclusive prefix sums over the batch of the labels below k0 and of the samples
        int cbs = ei > si ? c0 - si : 0, ns = ei - si;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y1 = __shfl_up_sync(kFull, cbs, o), y2 = __shfl_up_sync(kFull, ns, o);
            if (lane >= o) {
                cbs += y1;
                ns += y2;
            }
        }
        const unsigned ne = __ballot_sync(kFull, ei > si);
        const int pos = __popc(ne & lt);
        unsigned spec = 0;  // staged positions of runs with differentiating labels
        if (ei > si) {
            ws.pre[pos] = make_int2(cbs, ns);
            if (L > 0) {
                spec = 1u << pos;
                ws.meta[pos] = make_int4(c0, L | ((L > kShflMax || multi) ? 0x10000 : 0), (int)M1, (int)M2);
                if (multi) ws.lbl[pos] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
        }
        spec = __reduce_or_sync(kFull, spec);
        const int cbt = __shfl_sync(kFull, cbs, 31), nt = __shfl_sync(kFull, ns, 31);
        if (jn < U) {
            nf0 = __ldg(lab + na0);
            nl0 = __ldg(lab + nb0 - 1);
        }
        __syncwarp();
        const int cnt = __popc(ne);
        int r = 0;
        for (;;) {
            const int nxt = spec ? __ffs(spec) - 1 : cnt;
#pragma unroll 4
            for (; r < nxt; r++) {
                const int2 p = ws.pre[r];
                if (WIDE) {
                    const int64_t f = K + H * (int64_t)p.x - a * (int64_t)p.y;
                    const uint64_t af = (uint64_t)(f < 0 ? -f : f);
                    mx = af > mx ? af : mx;
                } else {
                    const int32_t f = (int32_t)(K + H * (uint32_t)p.x - a * (uint32_t)p.y);
                    mx32 = max(mx32, (uint32_t)(f < 0 ? -f : f));
                }
            }
            if (nxt >= cnt) break;
            // a run with differentiating labels: this lane's count of them below its k
            const int4 mt = ws.meta[nxt];
            const int Lr = mt.y & 0xffff;
            uint32_t add;
            if (!(mt.y >> 16)) {
                add = (uint32_t)(__popc((unsigned)mt.z & lt) + __popc((unsigned)mt.w & lt));
            } else if (Lr <= kShflMax) {
                const uint4 lb4 = ws.lbl[nxt];
                const uint32_t w4[4] = {lb4.x, lb4.y, lb4.z, lb4.w};
                add = 0;
#pragma unroll
                for (int t = 0; t < 4; t++)
                    add += (uint32_t)((int)(w4[t] & 0xffffu) < k) + (uint32_t)((int)(w4[t] >> 16) < k);
            } else if (Lr <= 32) {
                // histogram of the slice's labels over the 32 lanes, then an exclusive scan
                const int bin = lane < Lr ? (int)__ldg(lab + mt.x + lane) - k0 : -1;
                if (bin >= 0) atomicAdd(&ws.hist[bin], 1);
                __syncwarp();
                const int hv = ws.hist[lane];
                int incl = hv;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += y;
                }
                add = (uint32_t)(incl - hv);
                __syncwarp();
                if (bin >= 0) ws.hist[bin] = 0;
                __syncwarp();
            } else {
                add = (uint32_t)(lower_bound_lab(lab, mt.x, mt.x + Lr, k) - mt.x);
            }
            K += H * (Acc)add;
            const int2 p = ws.pre[nxt];
            if (WIDE) {
                const int64_t f = K + H * (int64_t)p.x - a * (int64_t)p.y;
                const uint64_t af = (uint64_t)(f < 0 ? -f : f);
                mx = af > mx ? af : mx;
            } else {
                const int32_t f = (int32_t)(K + H * (uint32_t)p.x - a * (uint32_t)p.y);
                mx32 = max(mx32, (uint32_t)(f < 0 ? -f : f));
            }
            r = nxt + 1;
            spec &= spec - 1;
        }
        K += H * (Acc)cbt - a * (Acc)nt;
        nonempty += cnt;
        __syncwarp();
    }
    g_out = WIDE ? mx : (uint64_t)mx32;
}

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

// ---------------------------------------------------------------- grid columns and gap bounds

// Exact columns at this lane's grid split gk (gk < 0: inactive lane) and, with the next
// lane's split gn, a bound over the gap.  With f_k(x) = H c_L^k(x) - (k - lo) C(x),
// D = Delta(x) = c_L^gn - c_L^gk, N = m H, and the fact that a step holds m samples
// (0 <= c_L^k - c_L^gk <= m (k - gk), 0 <= c_L^gn - c_L^k <= m (gn - k)), every split k in
// [gk, gn] satisfies, for every x,
//   m f_k in [m f_gk - ((gn - gk) m - D) C,  m f_gk + D (N - C)]     (from the left end)
//   m f_k in [m f_gn - D (N - C),  m f_gn + ((gn - gk) m - D) C]     (from the right end)
// (the extremes of H (c_L^k - c_L^gk) - (k - gk) C over the admissible c_L^k).  The larger
// modulus of the intersected interval, maximised over x, bounds m g_k over the gap.
__device__ __noinline__ void scan_grid(const uint16_t *__restrict__ lab, const int32_t *__restrict__ rt, int U,
                                       int T, int lo, int hi, int m, int gk, int gn, SliceStage<1> &st,
                                       uint64_t &g_out, uint64_t &ubm_out, int &nonempty) {
    const int lane = threadIdx.x & 31;
    const int64_t H = hi - lo, M = m, N = M * H, w = (int64_t)(gn - gk) * M;
    const int64_t a = gk - lo, an = gn - lo;
    int64_t cl = 0, C = 0;
    uint64_t mx = 0, ub = 0;
    nonempty = 0;
    // run bounds and end labels of the next batch are loaded one batch ahead (as in scan_slice1)
    int na0 = 0, nb0 = 0, nf0 = 0, nl0 = 0;
    if (lane < U) {
        na0 = __ldg(rt + lane);
        nb0 = __ldg(rt + lane + 1);
        nf0 = __ldg(lab + na0);
        nl0 = __ldg(lab + nb0 - 1);
    }
    for (int j0 = 0; j0 < U; j0 += 32) {
        const int j = j0 + lane;
        int si = 0, ei = 0, fi = 0, la = 0;
        const int a0 = na0, b0 = nb0, f0 = nf0, l0 = nl0;
        const int jn = j + 32;
        if (jn < U) {
            na0 = __ldg(rt + jn);
            nb0 = __ldg(rt + jn + 1);
        }
        if (j < U) {
            si = (f0 >= lo) ? a0 : (l0 < lo ? b0 : lower_bound_lab(lab, a0, b0, lo));
            ei = (l0 < hi) ? b0 : (f0 >= hi ? a0 : lower_bound_lab(lab, si, b0, hi));
            if (ei > si) {
                fi = (si == a0) ? f0 : __ldg(lab + si);
                la = (ei == b0) ? l0 : __ldg(lab + ei - 1);
            }
        }
        const unsigned ne = __ballot_sync(kFull, ei > si);
        if (ei > si) {
            const int pos = __popc(ne & lanemask_lt());
            st.si[pos] = si;
            st.ei[pos] = ei;
            st.cb[0][pos] = fi;
            st.cb[1][pos] = la;
        }
        if (jn < U) {
            nf0 = __ldg(lab + na0);
            nl0 = __ldg(lab + nb0 - 1);
        }
        __syncwarp();
        const int cnt = __popc(ne);
        for (int r = 0; r < cnt; r++) {
            const int rsi = st.si[r], rei = st.ei[r];
            C += rei - rsi;
            if (gk >= 0) cl += count_below(lab, rsi, rei, st.cb[0][r], st.cb[1][r], rsi, gk) - rsi;
            const int64_t cn = __shfl_down_sync(kFull, cl, 1);
            const int64_t f = H * cl - a * C;
            const uint64_t af = (uint64_t)(f < 0 ? -f : f);
            mx = af > mx ? af : mx;
            const int64_t fn = H * cn - an * C;
            const int64_t dl = cn - cl;
            const int64_t up = min(M * f + dl * (N - C), M * fn + (w - dl) * C);
            const int64_t dn = max(M * f - (w - dl) * C, M * fn - dl * (N - C));
            const uint64_t au = max((uint64_t)(up < 0 ? -up : up), (uint64_t)(dn < 0 ? -dn : dn));
            ub = au > ub ? au : ub;
        }
        nonempty += cnt;
        __syncwarp();
    }
    g_out = mx;
    ubm_out = ub;
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

// ---------------------------------------------------------------- run sweep
//
// The same g_k for every split of a segment, by one warp walking the splits in order.  The
// segment's runs with in-segment samples are numbered c = 0 .. U'-1 in value order, and for
// split k (a = k - lo)
//     v_k(c) = H c_L(x_c) - a C(x_c) = sum_{c' <= c} l_k(c') - a C_c,
// with l_k(c') = H times the left samples of run c' and C_c the in-segment samples of runs
// up to c.  Going from split k to k + 1 moves the m samples of step k to the left part: each
// adds H to l at its own run (the run index of every sample comes from the sort), so an
// update costs O(m), and the values at all runs follow from one pass over l.
//
// Lane L owns the block of R consecutive runs [L R, L R + R), R = ceil(U' / 32) rounded up to
// a multiple of 8, so that every lane walks the same number of runs in pairs of 16-byte loads
// and needs no per-run or per-load bounds test; positions at or past U' hold l = 0 and C = N (= m H), which repeat the value
// at the last run, v_k(U' - 1) = H m a - a m H = 0.  Within the block the lane accumulates
// the values relative to the run before the block,
//     v_k(c) - v_k(L R - 1) = sum_{L R <= c' <= c} l_k(c') - a (C_c - C_{L R - 1}),
// a sum over the block's samples of H (left) or 0, minus a each, so below m H^2 in magnitude,
// and keeps their max and min.  The block's own sum of l, scanned across the warp, then
// gives v_k(L R - 1) and so the block's true max and min; the warp maximum of the moduli is
// g_k.  The sweep takes segments with m H^2 < 2^31, where every quantity above is an exact
// 32-bit integer.
//
// Layout: the l of lane L's block sits at words [L Rs, L Rs + R) of the stage, Rs = R + 4; a
// lane reads its block four runs at a time (16-byte loads), and with Rs = 4 mod 8 the eight
// lanes of a quarter warp start on eight different four-bank groups, so the loads are free of
// bank conflicts.  Each lane keeps its block's C in registers (they do not change during a
// segment's sweep).
constexpr int kSweepMaxR = 48;                       // ceil(kSweepMaxRuns / 32), a multiple of 8
constexpr int kSweepLWords = 32 * (kSweepMaxR + 4);  // largest padded layout
// The evaluation loads a lane's next two quads before it knows whether its block has them: the
// last lane reads up to 4 words past the layout, into this tail (values never used).
constexpr int kSweepLTail = 16;
static_assert(kSweepMaxRuns <= 32 * kSweepMaxR && kSweepMaxR % 8 == 0, "lane blocks of kSweepMaxR runs");

struct __align__(16) SweepStage {
    uint32_t l[kSweepLWords + kSweepLTail];  // setup: count of series run r, then C of compact run c; sweep: l by layout position
    uint16_t map[kSweepMaxRuns];  // series run -> layout position of its compact run
};

union __align__(16) WarpSmem {
    WarpStage ws;
    SweepStage ss;
};

__device__ __forceinline__ bool sweepable(const RunParams &P, const SeriesDesc &d, int H) {
    return P.rk != nullptr && d.nruns <= kSweepMaxRuns && (uint64_t)d.m * (uint64_t)H * (uint64_t)H < (1ull << 31);
}

// Scan tile in effect for a segment of H steps: the series' tile, or for run-sweep series
// the sweep where the segment qualifies and single 32-split slices where it does not.
__device__ __forceinline__ int eff_kpt(const RunParams &P, const SeriesDesc &d, int H) {
    return d.kpt ? d.kpt : (sweepable(P, d, H) ? 0 : 1);
}

// l[map[r]] += w for every active lane.  A shared-memory reduction without return: the warp
// does not wait for it, and lanes that hit the same run are serialised by the hardware.
__device__ __forceinline__ void lc_add(SweepStage &ss, uint32_t r, uint32_t w, bool act) {
    if (act) atomicAdd(&ss.l[ss.map[r]], w);
}

// Run indices of one step held per lane between splits.  Vector form (series offset and m
// multiples of 4, so a step's row is 8-byte aligned): lane L holds samples 4L .. 4L + 3 of
// the step's first 128 as one 8-byte load.  Scalar form: samples L + 32 q, q < 4.
template <bool VEC>
struct StepBuf {
    uint32_t v[VEC ? 2 : 4];
};

template <bool VEC>
__device__ __forceinline__ void sweep_load_step(const uint16_t *__restrict__ rk, int64_t t, int m, int lane,
                                                StepBuf<VEC> &buf) {
    const uint16_t *src = rk + t * (int64_t)m;
    if constexpr (VEC) {
        uint2 x = make_uint2(0u, 0u);
        if (4 * lane < m) x = __ldg(reinterpret_cast<const uint2 *>(src) + lane);
        buf.v[0] = x.x;
        buf.v[1] = x.y;
    } else {
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int j = lane + 32 * q;
            buf.v[q] = (32 * q < m && j < m) ? (uint32_t)__ldg(src + j) : 0u;
        }
    }
}

// Move the samples of step t to the left part: l grows by H at each sample's run.  `buf`
// holds the step's first 128 run indices (sweep_load_step); the rest are read here.
template <bool VEC>
__device__ __forceinline__ void sweep_apply_step(SweepStage &ss, const uint16_t *__restrict__ rk, int64_t t, int m,
                                                 uint32_t H, int lane, const StepBuf<VEC> &buf) {
    const uint16_t *src = rk + t * (int64_t)m;
    if constexpr (VEC) {
        const bool act = 4 * lane < m;
        lc_add(ss, buf.v[0] & 0xffffu, H, act);
        lc_add(ss, buf.v[0] >> 16, H, act);
        lc_add(ss, buf.v[1] & 0xffffu, H, act);
        lc_add(ss, buf.v[1] >> 16, H, act);
        for (int j0 = 128; j0 < m; j0 += 128) {
            const bool a2 = j0 + 4 * lane < m;
            uint2 x = make_uint2(0u, 0u);
            if (a2) x = __ldg(reinterpret_cast<const uint2 *>(src + j0) + lane);
            lc_add(ss, x.x & 0xffffu, H, a2);
            lc_add(ss, x.x >> 16, H, a2);
            lc_add(ss, x.y & 0xffffu, H, a2);
            lc_add(ss, x.y >> 16, H, a2);
        }
    } else {
#pragma unroll
        for (int q = 0; q < 4; q++)
            if (32 * q < m) lc_add(ss, buf.v[q], H, lane + 32 * q < m);
        for (int j0 = 128; j0 < m; j0 += 32) {
            const bool act = j0 + lane < m;
            lc_add(ss, act ? (uint32_t)__ldg(src + j0 + lane) : 0u, H, act);
        }
    }
}

// Move the samples of steps [t0, t1) to the left part: their run indices are contiguous, so
// they are read as one range, 8 loads in flight per lane (8-byte loads in the vector form, 1024
// samples a round; else 2-byte loads, 256 a round).  Few registers: the lane block's C values
// stay live in registers around it (16 loads in flight make the learned kernels spill).
template <bool VEC>
__device__ void sweep_move_range(SweepStage &ss, const uint16_t *__restrict__ rk, int64_t t0, int64_t t1, int m,
                                 uint32_t H, int lane) {
    const int64_t f0 = t0 * m, e1 = t1 * m;
    if constexpr (VEC) {
        const uint2 *src = reinterpret_cast<const uint2 *>(rk);
        for (int64_t e0 = f0; e0 < e1; e0 += 1024) {
            uint2 x8[8];
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const int64_t e = e0 + 128 * q + 4 * lane;
                x8[q] = e < e1 ? __ldg(src + (e >> 2)) : make_uint2(0u, 0u);
            }
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const bool act = e0 + 128 * q + 4 * lane < e1;
                lc_add(ss, x8[q].x & 0xffffu, H, act);
                lc_add(ss, x8[q].x >> 16, H, act);
                lc_add(ss, x8[q].y & 0xffffu, H, act);
                lc_add(ss, x8[q].y >> 16, H, act);
            }
        }
    } else {
        for (int64_t e0 = f0; e0 < e1; e0 += 256) {
            uint32_t r8[8];
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const int64_t e = e0 + 32 * q + lane;
                r8[q] = e < e1 ? (uint32_t)__ldg(rk + e) : 0u;
            }
#pragma unroll
            for (int q = 0; q < 8; q++) lc_add(ss, r8[q], H, e0 + 32 * q + lane < e1);
        }
    }
}

// Four runs of a lane's block: running l sum hc, values hc - a C relative to the run before
// the block, their max and min (two-input max / min: the three-input intrinsics ran slower).
__device__ __forceinline__ void sweep_eval4(const uint4 q, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            uint32_t na, uint32_t &hc, int32_t &mx, int32_t &mn) {
    hc += q.x;
    const int32_t v0 = (int32_t)(hc + na * c0);
    hc += q.y;
    const int32_t v1 = (int32_t)(hc + na * c1);
    mx = max(mx, max(v0, v1));
    mn = min(mn, min(v0, v1));
    hc += q.z;
    const int32_t v2 = (int32_t)(hc + na * c2);
    hc += q.w;
    const int32_t v3 = (int32_t)(hc + na * c3);
    mx = max(mx, max(v2, v3));
    mn = min(mn, min(v2, v3));
}

// Best split (k, g) over A <= k <= B of segment [lo, hi) of a run-sweep series (A > lo: the
// samples of steps lo .. A - 1 are moved left first); every lane gets it.  `nonempty` = U', the
// runs with in-segment samples; `nev` = the splits evaluated.
//
// How the run sweep walks the splits: every split in order (kWalkAll); exact bound skipping
// (kWalkSkip); only the window splits of a window-only learned scan (kWalkWindows, for items
// with `win`, else every split).
constexpr int kWalkAll = 0, kWalkSkip = 1, kWalkWindows = 2;

// kWalkSkip: exact bound skipping.  Moving one step's m samples changes every v(c) by H s(c) - C(c),
// s(c) <= m and C(c) <= m H, so |g_{k+j} - g_k| <= j m H.  A split whose bound from the last
// evaluated split e, g_e + (k - e) m H, gives a D strictly below the best D found so far,
//     (g_e + (k - e) m H) a_b (H - a_b) < g_b a_k (H - a_k)        (64-bit products: m H^2 < 2^31),
// can be neither the argmax nor tie with it, so it is not evaluated; its samples still move.
// Window-only learned scan (MT4G_OPT_LEARNED_WINDOWS): split k of series `series` is a
// candidate when |k - c| <= half for one of its window centres c (c < 0: no window).
// The first window split in [A, B]; B + 1 when there is none.
__device__ __forceinline__ int first_window_split(const RunParams &P, int series, int A, int B) {
    const int32_t *c = P.win_center + (int64_t)series * P.n_win;
    int first = B + 1;
    for (int w = 0; w < P.n_win; w++) {
        const int cw = __ldg(c + w);
        if (cw < 0) continue;
        const int a = max(A, cw - P.half), b = min(B, cw + P.half);
        if (a <= b && a < first) first = a;
    }
    return first;
}

// The first merged window interval [a, b] of series `series` within [from, B]: a is the first
// window split >= from, b the end of the union of the windows that overlap or touch [a, b].
// False when no window split is left.  Every lane computes the same.
__device__ __forceinline__ bool window_interval(const RunParams &P, int series, int from, int B, int &a, int &b) {
    a = first_window_split(P, series, from, B);
    if (a > B) return false;
    const int32_t *c = P.win_center + (int64_t)series * P.n_win;
    b = a;
    for (bool grew = true; grew;) {
        grew = false;
        for (int w = 0; w < P.n_win; w++) {
            const int cw = __ldg(c + w);
            if (cw < 0) continue;
            const int lw = cw - P.half, hw = min(B, cw + P.half);
            if (lw <= b + 1 && hw > b) {
                b = hw;
                grew = true;
            }
        }
    }
    return true;
}

// FUSE: the previous split's scan inside the next split's evaluation (evaluate_fin); 1.6% faster
// in the plain kernels, 0.6% slower in the learned ones, whose routing code leaves less room.
template <bool VEC, int WALK, bool FUSE>
__device__ void sweep_best(const RunParams &P, const SeriesDesc &d, int lo, int hi, int A, int B, SweepStage &ss,
                           int &bk, uint64_t &bg, int &nonempty, int &nev, bool win = false, int series = 0) {
    const int lane = threadIdx.x & 31;
    const int U = d.nruns, m = d.m;
    const uint16_t *__restrict__ rk = P.rk + d.off;
    const uint32_t H = (uint32_t)(hi - lo);
    const unsigned lt = lanemask_lt();

    // in-segment samples per series run, into l[r]
    if (lo == 0 && hi == d.T) {
        const int32_t *rt = P.runs + d.run_base;
        for (int r = lane; r < U; r += 32) ss.l[r] = (uint32_t)(__ldg(rt + r + 1) - __ldg(rt + r));
    } else {
        for (int r = lane; r < U; r += 32) ss.l[r] = 0;
        __syncwarp();
        const int64_t e1 = (int64_t)hi * m;
        if constexpr (VEC) {  // rows are 8-byte aligned: four run indices per load, 2048 per round
            // the next round's loads are issued before the current round is counted
            const uint2 *src = reinterpret_cast<const uint2 *>(rk);
            uint2 x8[16], y8[16];
            const int64_t f0 = (int64_t)lo * m;
#pragma unroll
            for (int q = 0; q < 16; q++) {
                const int64_t e = f0 + 128 * q + 4 * lane;
                x8[q] = e < e1 ? __ldg(src + (e >> 2)) : make_uint2(0u, 0u);
            }
            for (int64_t e0 = f0; e0 < e1; e0 += 2048) {
#pragma unroll
                for (int q = 0; q < 16; q++) {
                    const int64_t e = e0 + 2048 + 128 * q + 4 * lane;
                    y8[q] = e < e1 ? __ldg(src + (e >> 2)) : make_uint2(0u, 0u);
                }
#pragma unroll
                for (int q = 0; q < 16; q++) {
                    const bool act = e0 + 128 * q + 4 * lane < e1;
                    if (act) {
                        atomicAdd(&ss.l[x8[q].x & 0xffffu], 1u);
                        atomicAdd(&ss.l[x8[q].x >> 16], 1u);
                        atomicAdd(&ss.l[x8[q].y & 0xffffu], 1u);
                        atomicAdd(&ss.l[x8[q].y >> 16], 1u);
                    }
                    x8[q] = y8[q];
                }
            }
        } else {
            for (int64_t e0 = (int64_t)lo * m; e0 < e1; e0 += 512) {  // 16 loads in flight per lane
                uint32_t r16[16];
#pragma unroll
                for (int q = 0; q < 16; q++) {
                    const int64_t e = e0 + 32 * q + lane;
                    r16[q] = e < e1 ? (uint32_t)__ldg(rk + e) : 0u;
                }
#pragma unroll
                for (int q = 0; q < 16; q++)
                    if (e0 + 32 * q + lane < e1) atomicAdd(&ss.l[r16[q]], 1u);
            }
        }
    }
    __syncwarp();
    // compaction, 128 runs per round (four consecutive runs per lane, one 16-byte load): a run's
    // compact slot is never above its own index, and every round reads its counts before it
    // writes, so the later rounds' counts survive.  Absent runs keep a stale map entry; no
    // sample of the segment refers to them.
    uint32_t nc = 0, cs = 0;  // runs kept so far, in-segment samples so far
    for (int r0 = 0; r0 < U; r0 += 128) {
        const int rb = r0 + 4 * lane;
        const uint4 q = *reinterpret_cast<const uint4 *>(&ss.l[rb]);  // within the stage (U <= 1536)
        const uint32_t n0 = rb < U ? q.x : 0u, n1 = rb + 1 < U ? q.y : 0u;
        const uint32_t n2 = rb + 2 < U ? q.z : 0u, n3 = rb + 3 < U ? q.w : 0u;
        const uint32_t s1 = n0 + n1, s2 = s1 + n2, s3 = s2 + n3;
        const unsigned k0 = __ballot_sync(kFull, n0 != 0), k1 = __ballot_sync(kFull, n1 != 0);
        const unsigned k2 = __ballot_sync(kFull, n2 != 0), k3 = __ballot_sync(kFull, n3 != 0);
        uint32_t incl = s3;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        __syncwarp();
        const uint32_t below = cs + incl - s3;  // in-segment samples of the runs before rb
        uint32_t ci = nc + (uint32_t)(__popc(k0 & lt) + __popc(k1 & lt) + __popc(k2 & lt) + __popc(k3 & lt));
        if (n0 != 0) {
            ss.map[rb] = (uint16_t)ci;
            ss.l[ci++] = below + n0;  // C of compact run ci, until the lanes have read it
        }
        if (n1 != 0) {
            ss.map[rb + 1] = (uint16_t)ci;
            ss.l[ci++] = below + s1;
        }
        if (n2 != 0) {
            ss.map[rb + 2] = (uint16_t)ci;
            ss.l[ci++] = below + s2;
        }
        if (n3 != 0) {
            ss.map[rb + 3] = (uint16_t)ci;
            ss.l[ci] = below + s3;
        }
        nc += (uint32_t)(__popc(k0) + __popc(k1) + __popc(k2) + __popc(k3));
        cs += __shfl_sync(kFull, incl, 31);
        __syncwarp();
    }
    const int Uc = (int)nc;
    const uint32_t N = cs;  // m H
    nonempty = Uc;
    int R = (Uc + 31) >> 5;
    R = max(8, (R + 7) & ~7);
    const int Rs = R + 4;
    const int nq = R >> 2;  // quads per block
    const int b0 = lane * R;
    const uint32_t Cb = b0 == 0 ? 0u : (b0 <= Uc ? ss.l[b0 - 1] : N);  // in-segment samples below the block
    uint32_t Cr[kSweepMaxR];
#pragma unroll
    for (int i = 0; i < kSweepMaxR / 4; i++) {  // 16-byte loads (b0 is a multiple of 8), within the stage
        const uint4 q = *reinterpret_cast<const uint4 *>(&ss.l[b0 + 4 * i]);
        Cr[4 * i] = b0 + 4 * i < Uc ? q.x : N;  // registers past R are never read
        Cr[4 * i + 1] = b0 + 4 * i + 1 < Uc ? q.y : N;
        Cr[4 * i + 2] = b0 + 4 * i + 2 < Uc ? q.z : N;
        Cr[4 * i + 3] = b0 + 4 * i + 3 < Uc ? q.w : N;
    }
    __syncwarp();
    // compact index -> layout position ci + 4 floor(ci / R); with R = 8 d (d <= 6) and
    // ci < 1536, floor(ci / R) = ((ci >> 3) (2^16 / d + 1)) >> 16 exactly
    const uint32_t magic = 65536u / (uint32_t)(R >> 3) + 1u;
    for (int r = lane; r < U; r += 32) {
        const uint32_t ci = ss.map[r];
        ss.map[r] = (uint16_t)(ci + 4u * (((ci >> 3) * magic) >> 16));
    }
    for (int w = 4 * lane; w < 32 * Rs; w += 128) *reinterpret_cast<uint4 *>(&ss.l[w]) = make_uint4(0u, 0u, 0u, 0u);
    __syncwarp();

    sweep_move_range<VEC>(ss, rk, lo, A, m, H, lane);
    const uint4 *lq = reinterpret_cast<const uint4 *>(&ss.l[lane * Rs]);
    // run indices two steps ahead (global loads in flight over two splits); the layout
    // positions of step k's samples are looked up at the top of split k and used by its moves
    // at the end, so the lookups' latency is spent under the evaluation
    bk = kNoK;
    bg = 0;
    uint32_t gk = 0;  // g of split kb + lane
    int kb = A;
    // The results of split k - 1 (block sum, relative max and min, a C below the block) are
    // finished in iteration k: a warp scan of the block sums, the block's true max and min, the
    // warp maximum of the moduli, and the argmax.  With FUSE (the plain kernels) this runs inside
    // the first group of split k's evaluation (evaluate_fin), else just before it (finish); the
    // last split of a range is finished after the loop.
    uint32_t p_blk = 0, p_h0 = 0;
    int32_t p_mx = 0, p_mn = 0;
    auto split_g = [&]() {
        uint32_t incl = p_blk;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t vs = (incl - p_blk) - p_h0;  // v at the run before the block
        const int32_t bmax = (int32_t)(vs + (uint32_t)p_mx), bmin = (int32_t)(vs + (uint32_t)p_mn);
        const uint32_t gl = (uint32_t)max(bmax, -bmin);  // max |v| over the block (bmin <= bmax)
        return __reduce_max_sync(kFull, gl);
    };
    // without skipping the argmax is taken 32 splits at a time (lane j holds split kb + j);
    // kend ends the current range of consecutive splits
    auto finish = [&](int kp, int kend) {
        const uint32_t g = split_g();
        if (lane == kp - kb) gk = g;
        if (kp - kb == 31 || kp == kend) {
            const int kk = kb + lane;
            if (kk <= kp && better(kk, (uint64_t)gk, bk, bg, lo, hi)) {
                bk = kk;
                bg = gk;
            }
            kb = kp + 1;
        }
    };
    // evaluate split k with the finish of split kp (= k - 1) interleaved into its first group of
    // quads, which every block has, so that the scan's shuffles overlap the evaluation
    auto evaluate_fin = [&](int k, int kp, int kend) {
        const uint32_t pb = p_blk, ph = p_h0;
        const int32_t pmx = p_mx, pmn = p_mn;
        const uint32_t a = (uint32_t)(k - lo), na = 0u - a;
        const uint32_t h0 = a * Cb;
        uint32_t hc = h0;
        int32_t mx = INT_MIN, mn = INT_MAX;
        uint4 q0 = lq[0], q1 = lq[1];
        uint32_t incl = pb;
        {
            const uint4 n0 = lq[2], n1 = lq[3];
            uint32_t y = __shfl_up_sync(kFull, incl, 1);
            if (lane >= 1) incl += y;
            sweep_eval4(q0, Cr[0], Cr[1], Cr[2], Cr[3], na, hc, mx, mn);
            y = __shfl_up_sync(kFull, incl, 2);
            if (lane >= 2) incl += y;
            sweep_eval4(q1, Cr[4], Cr[5], Cr[6], Cr[7], na, hc, mx, mn);
            y = __shfl_up_sync(kFull, incl, 4);
            if (lane >= 4) incl += y;
            y = __shfl_up_sync(kFull, incl, 8);
            if (lane >= 8) incl += y;
            y = __shfl_up_sync(kFull, incl, 16);
            if (lane >= 16) incl += y;
            q0 = n0;
            q1 = n1;
        }
        const uint32_t vs = (incl - pb) - ph;  // split kp: v at the run before the block
        const int32_t bmax = (int32_t)(vs + (uint32_t)pmx), bmin = (int32_t)(vs + (uint32_t)pmn);
        const uint32_t g = __reduce_max_sync(kFull, (uint32_t)max(bmax, -bmin));
#pragma unroll
        for (int gg = 1; gg < kSweepMaxR / 8; gg++) {
            if (2 * gg >= nq) break;
            const uint4 n0 = lq[2 * gg + 2], n1 = lq[2 * gg + 3];
            sweep_eval4(q0, Cr[8 * gg], Cr[8 * gg + 1], Cr[8 * gg + 2], Cr[8 * gg + 3], na, hc, mx, mn);
            sweep_eval4(q1, Cr[8 * gg + 4], Cr[8 * gg + 5], Cr[8 * gg + 6], Cr[8 * gg + 7], na, hc, mx, mn);
            q0 = n0;
            q1 = n1;
        }
        if (lane == kp - kb) gk = g;
        if (kp - kb == 31 || kp == kend) {
            const int kk = kb + lane;
            if (kk <= kp && better(kk, (uint64_t)gk, bk, bg, lo, hi)) {
                bk = kk;
                bg = gk;
            }
            kb = kp + 1;
        }
        p_blk = hc - h0;
        p_h0 = h0;
        p_mx = mx;
        p_mn = mn;
    };
    // the values of split k into p_blk, p_h0, p_mx, p_mn (l holds the left counts of split k)
    auto evaluate = [&](int k) {
        const uint32_t a = (uint32_t)(k - lo), na = 0u - a;
        const uint32_t h0 = a * Cb;
        uint32_t hc = h0;
        int32_t mx = INT_MIN, mn = INT_MAX;
        uint4 q0 = lq[0], q1 = lq[1];
        // the block in groups of two quads (nq is even), the next group's loads issued before the
        // current group is evaluated, whether or not the block has them (nq is the same for every
        // lane; the two quads after the block's last are loaded, within the stage, and not used)
#pragma unroll
        for (int g = 0; g < kSweepMaxR / 8; g++) {
            if (2 * g >= nq) break;
            const uint4 n0 = lq[2 * g + 2], n1 = lq[2 * g + 3];
            sweep_eval4(q0, Cr[8 * g], Cr[8 * g + 1], Cr[8 * g + 2], Cr[8 * g + 3], na, hc, mx, mn);
            sweep_eval4(q1, Cr[8 * g + 4], Cr[8 * g + 5], Cr[8 * g + 6], Cr[8 * g + 7], na, hc, mx, mn);
            q0 = n0;
            q1 = n1;
        }
        p_blk = hc - h0;  // sum of l over the block
        p_h0 = h0;
        p_mx = mx;
        p_mn = mn;
    };
    nev = 0;
    if constexpr (WALK == kWalkSkip) {
        // Exact bound skipping, pipelined like the full walk (run indices two steps ahead, every
        // step's samples moved after its split): split k is evaluated only when the bound from the
        // last evaluated split e, g_e + (k - e) m H, can reach the best D so far.  With
        // m H^2 < 2^31 both products of the test stay below 2^61.
        int e = kNoK;
        uint32_t ge = 0;
        bool pending = false;  // split e evaluated, its g not yet taken
        StepBuf<VEC> nxt, nxt2;
        sweep_load_step<VEC>(rk, A, m, lane, nxt);
        sweep_load_step<VEC>(rk, min(A + 1, B), m, lane, nxt2);
        const uint64_t mH = (uint64_t)m * H;
        for (int k = A; k <= B; k++) {
            const StepBuf<VEC> cur = nxt;
            uint32_t pos0 = 0, pos1 = 0, pos2 = 0, pos3 = 0;
            if (VEC) {  // lanes past the step's m samples look up run 0 and do not use it
                pos0 = ss.map[cur.v[0] & 0xffffu];
                pos1 = ss.map[cur.v[0] >> 16];
                pos2 = ss.map[cur.v[1] & 0xffffu];
                pos3 = ss.map[cur.v[1] >> 16];
            }
            nxt = nxt2;
            sweep_load_step<VEC>(rk, min(k + 2, B), m, lane, nxt2);
            if (pending) {
                ge = split_g();
                if (better(e, (uint64_t)ge, bk, bg, lo, hi)) {
                    bk = e;
                    bg = ge;
                }
                pending = false;
            }
            bool ev = true;
            if (e != kNoK) {
                const uint64_t ub = (uint64_t)ge + (uint64_t)(k - e) * mH;
                const uint64_t db = (uint64_t)(bk - lo) * (uint64_t)(hi - bk);
                const uint64_t dk = (uint64_t)(k - lo) * (uint64_t)(hi - k);
                ev = !(ub * db < (uint64_t)bg * dk);
            }
            // the barriers order the moves only around an evaluation: the moves of skipped splits
            // follow one another with none
            if (ev) {
                __syncwarp();
                nev++;
                evaluate(k);
                e = k;
                pending = true;
                __syncwarp();
            }
            if constexpr (VEC) {
                if (4 * lane < m) {
                    atomicAdd(&ss.l[pos0], H);
                    atomicAdd(&ss.l[pos1], H);
                    atomicAdd(&ss.l[pos2], H);
                    atomicAdd(&ss.l[pos3], H);
                }
                const uint16_t *src = rk + (int64_t)k * m;
                for (int j0 = 128; j0 < m; j0 += 128) {
                    const bool a2 = j0 + 4 * lane < m;
                    uint2 x = make_uint2(0u, 0u);
                    if (a2) x = __ldg(reinterpret_cast<const uint2 *>(src + j0) + lane);
                    lc_add(ss, x.x & 0xffffu, H, a2);
                    lc_add(ss, x.x >> 16, H, a2);
                    lc_add(ss, x.y & 0xffffu, H, a2);
                    lc_add(ss, x.y >> 16, H, a2);
                }
            } else {
                sweep_apply_step<VEC>(ss, rk, k, m, H, lane, cur);
            }
        }
        if (pending) {
            ge = split_g();
            if (better(e, (uint64_t)ge, bk, bg, lo, hi)) {
                bk = e;
                bg = ge;
            }
        }
        __syncwarp();
        return;
    }
    // every split of [Ai, Bi] in order, software-pipelined: run indices two steps ahead, split
    // k - 1 finished while split k's first loads are in flight; step k moves left after split k,
    // step Bi too (nothing reads l after the last split but the window walk, which goes on from
    // step Bi + 1), so that the loop has no per-split tests
    auto sweep_range = [&](int Ai, int Bi) {
        kb = Ai;
        StepBuf<VEC> nxt, nxt2;
        sweep_load_step<VEC>(rk, Ai, m, lane, nxt);
        sweep_load_step<VEC>(rk, min(Ai + 1, Bi), m, lane, nxt2);
        for (int k = Ai; k <= Bi; k++) {
            const StepBuf<VEC> cur = nxt;
            uint32_t pos0 = 0, pos1 = 0, pos2 = 0, pos3 = 0;
            if (VEC) {  // lanes past the step's m samples look up run 0 and do not use it
                pos0 = ss.map[cur.v[0] & 0xffffu];
                pos1 = ss.map[cur.v[0] >> 16];
                pos2 = ss.map[cur.v[1] & 0xffffu];
                pos3 = ss.map[cur.v[1] >> 16];
            }
            nxt = nxt2;
            sweep_load_step<VEC>(rk, min(k + 2, Bi), m, lane, nxt2);  // past Bi: a step of the segment, unused
            __syncwarp();
            nev++;
            if constexpr (FUSE) {
                evaluate_fin(k, k - 1, Bi);  // at k = Ai it records nothing (no lane has split kb - 1)
            } else {
                finish(k - 1, Bi);  // at k = Ai it records nothing (no lane has split kb - 1)
                evaluate(k);
            }
            // every lane has read l for split k: step k's samples move left now (reductions the warp
            // does not wait for)
            __syncwarp();
            {
                if constexpr (VEC) {
                    if (4 * lane < m) {
                        atomicAdd(&ss.l[pos0], H);
                        atomicAdd(&ss.l[pos1], H);
                        atomicAdd(&ss.l[pos2], H);
                        atomicAdd(&ss.l[pos3], H);
                    }
                    const uint16_t *src = rk + (int64_t)k * m;
                    for (int j0 = 128; j0 < m; j0 += 128) {
                        const bool a2 = j0 + 4 * lane < m;
                        uint2 x = make_uint2(0u, 0u);
                        if (a2) x = __ldg(reinterpret_cast<const uint2 *>(src + j0) + lane);
                        lc_add(ss, x.x & 0xffffu, H, a2);
                        lc_add(ss, x.x >> 16, H, a2);
                        lc_add(ss, x.y & 0xffffu, H, a2);
                        lc_add(ss, x.y >> 16, H, a2);
                    }
                } else {
                    sweep_apply_step<VEC>(ss, rk, k, m, H, lane, cur);
                }
            }
        }
        finish(Bi, Bi);
    };
    if (WALK == kWalkWindows && win) {
        // window-only scan: the merged window intervals within [A, B] (A is the first window
        // split, the steps before it moved in the setup); the steps between intervals move in one
        // pass each
        int from = A, prev = -1, a = 0, b = 0;
        while (window_interval(P, series, from, B, a, b)) {
            if (prev >= 0) {
                __syncwarp();
                sweep_move_range<VEC>(ss, rk, prev + 1, a, m, H, lane);  // steps prev + 1 .. a - 1
            }
            sweep_range(a, b);
            prev = b;
            from = b + 1;
        }
    } else {
        sweep_range(A, B);
    }
    warp_best(bk, bg, lo, hi);
    __syncwarp();
}

// Reserve `tot` queue slots and count them as pending (one lane).  Returns the first slot,
// or ~0 when the queue is full (then nothing is pending and the status says so).
__device__ unsigned long long reserve_slots(const RunParams &P, int tot) {
    atomicAdd((unsigned long long *)&P.q->pending, (unsigned long long)tot);
    const unsigned long long base = atomicAdd(&P.q->tail, (unsigned long long)tot);
    if (base + tot > P.q->cap) {
        atomicOr(&P.q->status, kStatusQueueFull);
        atomicAdd((unsigned long long *)&P.q->pending, (unsigned long long)(-(long long)tot));
        return ~0ull;
    }
    return base;
}

__device__ __forceinline__ void put_item(const RunParams &P, unsigned long long slot, const WorkItem &w) {
    int4 *dst = reinterpret_cast<int4 *>(P.items + slot);
    dst[0] = make_int4(w.series, w.lo, w.hi, w.chunk);
    dst[1] = make_int4(w.kind_nch, w.k0, w.klim, w.rec);
}

// The full scan of segment [lo, hi) (all lanes of a warp call it with the same arguments):
// run-sweep items where the sweep takes the segment, else its slices.  The sweep is cut into
// parts when fewer items are pending than the launch has warps (and the queue is at most half
// used), so that idle warps share a long segment.
// want_parts > 0 (the top level of a learned call): that many parts, as the host planned them.
__device__ void push_plain(const RunParams &P, const SeriesDesc &d, int series, int lo, int hi, uint32_t epoch,
                           int want_parts) {
    const int lane = threadIdx.x & 31;
    const int A = lo + P.min_seg, B = hi - P.min_seg;
    const int kpt = eff_kpt(P, d, hi - lo);
    int nch = 0;
    if (kpt == 0) {
        int want = want_parts;
        if (want_parts <= 0 && lane == 0) {
            want = 1;
            const long long pend = *(volatile const long long *)&P.q->pending;
            const unsigned long long tail = *(volatile const unsigned long long *)&P.q->tail;
            if (tail < P.q->cap / 2 && pend < (long long)P.sweep_warps)
                want = (int)(P.sweep_warps / (pend > 1 ? pend : 1));
        }
        nch = sweep_parts(hi - lo, P.min_seg, __shfl_sync(kFull, want, 0));
    } else {
        nch = seg_chunks(hi - lo, P.min_seg, kpt);
    }
    unsigned long long base = 0;
    if (lane == 0) base = reserve_slots(P, nch);
    base = __shfl_sync(kFull, base, 0);
    if (base == ~0ull) return;
    for (int c = lane; c < nch; c += 32) {
        if (kpt == 0) {
            int k0, k1;
            sweep_part_range(A, B, c, nch, k0, k1);
            put_item(P, base + c, WorkItem{series, lo, hi, c, kPlain | (nch << 8), k0, k1, kSweepItem});
        } else {
            put_item(P, base + c, WorkItem{series, lo, hi, c, kPlain | (nch << 8), 0, B, -1});
        }
    }
    if (lane == 0) P.gcount[base] = 0;
    __threadfence();
    for (int c = lane; c < nch; c += 32) st_release_u32((uint32_t *)P.ready + base + c, epoch);
}

// Window-only scan of a swept segment (MT4G_OPT_LEARNED_WINDOWS; all lanes, same arguments):
// its window splits, by the sweep.  A segment without any is a leaf, and a series without any at
// its top level takes the full scan.
__device__ __noinline__ void push_window_segment(const RunParams &P, const SeriesDesc &d, int series, int lo, int hi,
                                                 uint32_t epoch, int want_parts) {
    const int lane = threadIdx.x & 31;
    const int A = lo + P.min_seg, B = hi - P.min_seg;
    int fw = 0;
    if (lane == 0) fw = first_window_split(P, series, A, B);
    fw = __shfl_sync(kFull, fw, 0);
    if (fw > B) {
        if (lo != 0 || hi != d.T) return;
        if (lane == 0) {
            P.fallback[series] = 1;
            __threadfence();
        }
        __syncwarp();
    }
    push_plain(P, d, series, lo, hi, epoch, want_parts);
}

// Push the work for segment [lo, hi) (all lanes of a warp call it with the same arguments).
// Plain series, and learned segments with no window centred at least half/2 inside their
// splits: the full scan (push_plain).  Other learned segments: a probe group of the window
// slices that reach the segment's splits plus one grid item.
__device__ __noinline__ void push_segment(const RunParams &P, const SeriesDesc &d, int series, int lo, int hi, uint32_t epoch,
                                          int want_parts = 0) {
    const int lane = threadIdx.x & 31;
    const int A = lo + P.min_seg, B = hi - P.min_seg;
    if (B < A) return;
    const bool learned = P.mode == kRunLearned && !P.fallback[series];
    if (!learned) {
        push_plain(P, d, series, lo, hi, epoch, want_parts);
        return;
    }
    if (P.win_only && eff_kpt(P, d, hi - lo) == 0) {
        push_window_segment(P, d, series, lo, hi, epoch, want_parts);
        return;
    }
    // a probe only pays where a window is centred well inside the segment; elsewhere (in
    // particular the pieces between consecutive change points) the full scan decides
    int inner = 0;
    if (lane < P.n_win) {
        const int c = P.win_center[(int64_t)series * P.n_win + lane];
        inner = c >= A + P.half / 2 && c <= B - P.half / 2;
    }
    if (__ballot_sync(kFull, inner) == 0) {
        push_plain(P, d, series, lo, hi, epoch, want_parts);
        return;
    }
    if (lane == 0) {
        int ks[8];
        int nw = 0;
        for (int w = 0; w < P.n_win; w++) {
            const int c = P.win_center[(int64_t)series * P.n_win + w];
            if (c < 0) continue;
            const int k0 = c - P.half;
            if (k0 + 31 < A || k0 > B) continue;
            ks[nw++] = k0;
        }
        const int tot = nw + 1;
        const unsigned long long rec = atomicAdd(&P.q->rec_next, 1ull);
        if (rec >= P.q->rec_cap) {
            atomicOr(&P.q->status, kStatusQueueFull);
            return;
        }
        const unsigned long long base = reserve_slots(P, tot);
        if (base == ~0ull) return;
        for (int j = 0; j < nw; j++)
            put_item(P, base + j, WorkItem{series, lo, hi, j, kWindow | (tot << 8), ks[j], B, (int)rec});
        put_item(P, base + nw, WorkItem{series, lo, hi, nw, kGrid | (tot << 8), A, B, (int)rec});
        P.gcount[base] = 0;
        __threadfence();
        for (int j = 0; j < tot; j++) st_release_u32((uint32_t *)P.ready + base + j, epoch);
    }
    __syncwarp();
}

// Decide a segment whose best split is known exactly (all lanes, same arguments):
// p-value, outputs, and if significant the change point and the work for both parts.
__device__ __noinline__ void finish_segment(const RunParams &P, const SeriesDesc &d, int series, int lo, int hi, int k,
                               uint64_t g, uint32_t epoch) {
    const int lane = threadIdx.x & 31;
    int accept = 0, rescan = 0;
    if (lane == 0 && k == kNoK) {
        // a window-only segment without window splits (pushed only at the top level, by parts
        // whose ranges miss the windows): not significant
    } else if (lane == 0) {
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
            // Eq. 1: d_alpha = sqrt(-1/2 ln(alpha / 2) (n_L + n_R) / (n_L n_R)), products in this
            // order, each rounded once
            P.cp_crit[slot] = __dsqrt_rn(__ddiv_rn(__dmul_rn(P.crit_c, (double)N),
                                                   __dmul_rn((double)(m * a), (double)(m * b))));
            P.cp_flag[slot] = 1;
            accept = 1;
        }
    }
    if (lane == 0 && !accept && P.mode == kRunLearned && P.win_only && lo == 0 && hi == d.T &&
        !P.fallback[series] && eff_kpt(P, d, hi - lo) == 0) {
        // window-only top level without a significant split: the series falls back to the full scan
        P.fallback[series] = 1;
        __threadfence();
        rescan = 1;
    }
    accept = __shfl_sync(kFull, accept, 0);
    if (__shfl_sync(kFull, rescan, 0)) {
        push_segment(P, d, series, lo, hi, epoch);  // the series' flag now routes it to the full scan
        return;
    }
    if (!accept) return;
    push_segment(P, d, series, lo, k, epoch);
    push_segment(P, d, series, k, hi, epoch);
}


// After a learned segment's probe group: (k, g) is the best exact split among its windows
// and grid splits.  A gap (a, b) is certified when its bound cannot reach D(k):
//   ub * den(k) < g * min(den(a + 1), den(b - 1))   (den concave, so its minimum over the
// gap is at an end; strict, so an equal D further left cannot be missed).  All gaps
// certified: k is the argmax.  Otherwise, if D(k) is not significant and no gap's bound
// can be (p of the bound > alpha (1 + 1e-9), the margin covering FP64 rounding of Q),
// the segment is not split, exactly as the full scan would decide.  Otherwise the
// uncertified gaps are scanned by refine slices.
__device__ __noinline__ void certify_segment(const RunParams &P, const SeriesDesc &d, const WorkItem &it, int k, uint64_t g,
                                uint32_t epoch) {
    const int lane = threadIdx.x & 31;
    const int lo = it.lo, hi = it.hi;
    CertRecord *rec = P.recs + it.rec;
    const int n_gap = __ldcg(&rec->n_gap);
    const uint64_t dk = (uint64_t)(k - lo) * (uint64_t)(hi - k);
    bool open = false;  // this lane's gap is uncertified
    int ga = 0, gb = 0;
    uint64_t gub = 0, dmin = 1;
    if (lane < n_gap) {
        ga = __ldcg(&rec->a[lane]);
        gb = __ldcg(&rec->b[lane]);
        gub = __ldcg(&rec->ub[lane]);
        if (gb - ga > 1) {
            const uint64_t d1 = (uint64_t)(ga + 1 - lo) * (uint64_t)(hi - ga - 1);
            const uint64_t d2 = (uint64_t)(gb - 1 - lo) * (uint64_t)(hi - gb + 1);
            dmin = d1 < d2 ? d1 : d2;
            open = !prod_less(gub, dk, g, dmin);
        }
    }
    const unsigned openm = __ballot_sync(kFull, open);
    if (openm == 0) {
        if (lane == 0) atomicAdd(&P.q->certified, 1ull);
        finish_segment(P, d, it.series, lo, hi, k, g, epoch);
        return;
    }
    // not significant anywhere?
    const int64_t m = d.m, H = hi - lo;
    bool quiet = true;
    if (lane == 0) {
        const double pk = ks_pvalue(m * (int64_t)g, (m * (k - lo)) * (m * (hi - k)), m * H);
        quiet = pk > P.alpha;
    }
    if (open) {
        const uint64_t cap_f = (uint64_t)m * (uint64_t)H * (uint64_t)H / 4 + 1;  // |f| never exceeds m H^2 / 4
        const uint64_t u = gub < cap_f ? gub : cap_f;
        const double pu = ks_pvalue((int64_t)(m * (int64_t)u), (int64_t)(m * m) * (int64_t)dmin, m * H);
        quiet = quiet && pu > P.alpha * (1.0 + 1e-9);
    }
    if (__all_sync(kFull, quiet)) {
        if (lane == 0) atomicAdd(&P.q->certified, 1ull);
        return;
    }
    // refine the open gaps: consecutive open gaps form one range a + 1 .. b - 1 (the grid splits
    // between them are scanned again, which changes nothing), cut into slices of 32 splits, so
    // that narrow gaps do not leave most lanes of a slice idle
    const bool owner = open && (lane == 0 || !((openm >> (lane - 1)) & 1u));
    const unsigned after = lane < 31 ? ~openm & (0xffffffffu << (lane + 1)) : 0u;
    const int last = after ? __ffs(after) - 2 : 31;  // last open gap of this lane's run
    const int rb = __shfl_sync(kFull, gb, last);
    const int ns = owner ? (rb - ga - 1 + 31) / 32 : 0;
    int incl = ns;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const int tot = __shfl_sync(kFull, incl, 31);
    unsigned long long base = 0;
    if (lane == 0) {
        rec->best_k = k;
        rec->best_g = g;
        atomicAdd(&P.q->refined, 1ull);
        base = reserve_slots(P, tot);
    }
    base = __shfl_sync(kFull, base, 0);
    if (base == ~0ull) return;
    const int first = incl - ns;
    for (int i = 0; i < ns; i++)
        put_item(P, base + first + i,
                 WorkItem{it.series, lo, hi, first + i, kRefine | (tot << 8), ga + 1 + 32 * i, rb - 1, it.rec});
    if (lane == 0) P.gcount[base] = 0;
    __threadfence();
    for (int i = 0; i < ns; i++) st_release_u32((uint32_t *)P.ready + base + first + i, epoch);
}

// Scan one slice and reduce it to the warp's best (k, g) over kmin <= k <= kmax; every lane
// gets the result.
template <bool WIDE, int KPT>
__device__ void slice_best(const RunParams &P, const SeriesDesc &d, int lo, int hi, int k0, int kmin, int kmax,
                           WarpStage &stage, int &bk, uint64_t &bg, int &nonempty) {
    const int lane = threadIdx.x & 31;
    uint64_t g[KPT];
    if constexpr (KPT == 1) {
        scan_slice1<WIDE>(P.lab + d.off, P.runs + d.run_base, d.nruns, d.T, lo, hi, k0, stage, g[0], nonempty);
    } else {
        SliceStage<KPT> &st = *reinterpret_cast<SliceStage<KPT> *>(&stage.u);
        scan_slice<WIDE, KPT>(P.lab + d.off, P.runs + d.run_base, d.nruns, d.T, lo, hi, k0, st, g, nonempty);
    }
    bk = kNoK;
    bg = 0;
#pragma unroll
    for (int q = 0; q < KPT; q++) {
        const int k = k0 + 32 * q + lane;
        if (k >= kmin && k <= kmax && better(k, g[q], bk, bg, lo, hi)) {
            bk = k;
            bg = g[q];
        }
    }
    warp_best(bk, bg, lo, hi);
}

// Persistent kernel: every warp independently takes tickets from the queue and processes
// one item per ticket.  No block-level synchronisation.
// LEARNED = false compiles the plain-segmentation kernel without the probe, certification and
// refinement paths (fewer registers: no spills); learned calls launch the full one.
// SWEEP = true adds the run sweep: each warp's shared memory then holds a SweepStage (for
// up to kSweepMaxRuns runs), launched as CTAs of kSweepThreads; without it, the smaller
// slice staging allows more resident warps.
// WALK (with SWEEP) picks how the run sweep walks the splits: all of them, exact bound skipping
// (MT4G_OPT_SWEEP_SKIP), or window-only learned scans (MT4G_OPT_LEARNED_WINDOWS).
template <bool LEARNED, bool SWEEP, int WALK = kWalkAll>
__global__ void __launch_bounds__(SWEEP ? kSweepThreads : kScanThreads, SWEEP ? 8 : 4)
    queue_kernel(RunParams P, uint32_t epoch) {
    if (P.gate != kGateNone) {  // one of a learned call's two launches: the sort's count decides which
        const unsigned long long unswept = *(volatile const unsigned long long *)&P.q->unswept;
        if ((P.gate == kGateAllSwept) != (unswept == 0)) return;
    }
    using Smem = typename std::conditional<SWEEP, WarpSmem, WarpStage>::type;
    __shared__ Smem s_stage[(SWEEP ? kSweepThreads : kScanThreads) / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpStage &stage = *reinterpret_cast<WarpStage *>(&s_stage[warp]);
    const unsigned long long cap = P.q->cap;
    unsigned long long my_evals = 0, my_swept = 0;

    for (;;) {
        unsigned long long ticket = 0;
        int4 raw0 = make_int4(0, 0, 0, 0), raw1 = make_int4(0, 0, 0, 0);
        int state = 0;
        if (lane == 0) {
            ticket = atomicAdd(&P.q->head, 1ull);
            const unsigned long long t0 = globaltimer_ns();
            unsigned ns = 32;
            for (;;) {
                if (ticket < cap && ld_acquire_u32((const uint32_t *)P.ready + ticket) >= epoch) {
                    raw0 = __ldcg(reinterpret_cast<const int4 *>(P.items + ticket));
                    raw1 = __ldcg(reinterpret_cast<const int4 *>(P.items + ticket) + 1);
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
        const WorkItem it{__shfl_sync(kFull, raw0.x, 0), __shfl_sync(kFull, raw0.y, 0),
                          __shfl_sync(kFull, raw0.z, 0), __shfl_sync(kFull, raw0.w, 0),
                          __shfl_sync(kFull, raw1.x, 0), __shfl_sync(kFull, raw1.y, 0),
                          __shfl_sync(kFull, raw1.z, 0), __shfl_sync(kFull, raw1.w, 0)};
        const SeriesDesc d = P.desc[it.series];
        const int lo = it.lo, hi = it.hi;
        const int kind = item_kind(it), nch = item_nch(it);
        const int A = lo + P.min_seg, B = hi - P.min_seg;
        const uint64_t H = (uint64_t)(hi - lo);
        const bool wide = (uint64_t)d.m * H * H >= (1ull << 33);
        int nonempty = 0, bk = kNoK;
        uint64_t bg = 0;
        bool repushed = false;
        if (LEARNED && kind == kGrid) {
            const int ng = min(kMaxGrid, B - A + 1);
            const int gk = lane < ng ? (ng == 1 ? A : A + (int)((int64_t)lane * (B - A) / (ng - 1))) : -1;
            const int gn = __shfl_down_sync(kFull, gk, 1);
            uint64_t g = 0, ubm = 0;
            scan_grid(P.lab + d.off, P.runs + d.run_base, d.nruns, d.T, lo, hi, d.m, gk, lane + 1 < ng ? gn : gk,
                      stage.u.s1, g, ubm, nonempty);
            const uint64_t ub = (ubm + (uint64_t)d.m - 1) / (uint64_t)d.m;  // bound on g over the gap
            my_evals += (unsigned long long)ng * (unsigned long long)nonempty;
            CertRecord *rec = P.recs + it.rec;
            if (lane + 1 < ng) {
                rec->a[lane] = gk;
                rec->b[lane] = gn;
                rec->ub[lane] = ub;
            }
            if (lane == 0) rec->n_gap = ng - 1;
            bk = gk >= 0 ? gk : kNoK;
            bg = gk >= 0 ? g : 0;
            warp_best(bk, bg, lo, hi);
        } else if (SWEEP && kind == kPlain && it.rec == kSweepItem) {
            if constexpr (SWEEP) {
                if (eff_kpt(P, d, hi - lo) == 0) {
                    SweepStage &ss = *reinterpret_cast<SweepStage *>(&s_stage[warp]);
                    const bool vec = (d.off & 3) == 0 && (d.m & 3) == 0;
                    int nev = 0;
                    // window-only learned scan: evaluate only the item's window splits
                    bool win = false;
                    int k0 = it.k0;
                    if (LEARNED && WALK == kWalkWindows && P.win_only && P.mode == kRunLearned &&
                        *(volatile const int32_t *)(P.fallback + it.series) == 0) {
                        win = true;
                        k0 = first_window_split(P, it.series, it.k0, it.klim);
                    }
                    if (k0 > it.klim) {
                        bk = kNoK;  // no window split in this part's range
                        bg = 0;
                    } else if (vec) {
                        sweep_best<true, WALK, !LEARNED>(P, d, lo, hi, k0, it.klim, ss, bk, bg, nonempty, nev, win,
                                                         it.series);
                    } else {
                        sweep_best<false, WALK, !LEARNED>(P, d, lo, hi, k0, it.klim, ss, bk, bg, nonempty, nev, win,
                                                          it.series);
                    }
                    my_evals += (unsigned long long)nev * (unsigned long long)nonempty;
                    my_swept += it.chunk == 0;
                } else {
                    // a top-level item of a series planned for the sweep that it cannot take (too
                    // many distinct values, or a wide segment): the segment goes back to the queue
                    // as slices, once
                    if (it.chunk == 0) push_segment(P, d, it.series, lo, hi, epoch);
                    repushed = true;
                }
            }
        } else if (kind == kPlain) {
            const int kpt = eff_kpt(P, d, hi - lo);
            const int k0 = A + it.chunk * 32 * kpt;
            const int kmax = min(k0 + 32 * kpt - 1, B);
            if (kpt == 4) {
                if (wide) slice_best<true, 4>(P, d, lo, hi, k0, k0, kmax, stage, bk, bg, nonempty);
                else slice_best<false, 4>(P, d, lo, hi, k0, k0, kmax, stage, bk, bg, nonempty);
            } else if (kpt == 2) {
                if (wide) slice_best<true, 2>(P, d, lo, hi, k0, k0, kmax, stage, bk, bg, nonempty);
                else slice_best<false, 2>(P, d, lo, hi, k0, k0, kmax, stage, bk, bg, nonempty);
            } else {
                if (wide) slice_best<true, 1>(P, d, lo, hi, k0, k0, kmax, stage, bk, bg, nonempty);
                else slice_best<false, 1>(P, d, lo, hi, k0, k0, kmax, stage, bk, bg, nonempty);
            }
            my_evals += (unsigned long long)(kmax - k0 + 1) * (unsigned long long)nonempty;
        } else if (LEARNED) {  // window or refine slice: 32 explicit splits
            const int k0 = it.k0;
            const int kmin = max(k0, A), kmax = min(k0 + 31, min(it.klim, B));
            if (wide) slice_best<true, 1>(P, d, lo, hi, k0, kmin, kmax, stage, bk, bg, nonempty);
            else slice_best<false, 1>(P, d, lo, hi, k0, kmin, kmax, stage, bk, bg, nonempty);
            my_evals += (unsigned long long)max(0, kmax - kmin + 1) * (unsigned long long)nonempty;
        }

        if (repushed) {
            // nothing to record: the slices pushed above decide the segment
        } else if (nch == 1 && kind == kPlain) {
            finish_segment(P, d, it.series, lo, hi, bk, bg, epoch);
        } else {
            // write this member's result over its consumed slot; the last member combines
            const unsigned long long base = ticket - (unsigned long long)it.chunk;
            int last = 0;
            if (lane == 0) {
                *reinterpret_cast<ChunkResult *>(P.items + ticket) = ChunkResult{bk, 0, bg};
                __threadfence();
                const uint32_t old = atomicAdd(P.gcount + base, 1u);
                last = old == (uint32_t)nch - 1u;
            }
            last = __shfl_sync(kFull, last, 0);
            if (last) {
                __threadfence();
                int ck = kNoK;
                uint64_t cg = 0;
                for (int c = lane; c < nch; c += 32) {
                    const int4 r2 = __ldcg(reinterpret_cast<const int4 *>(P.items + base + c));
                    const uint64_t g2 = (uint64_t)(uint32_t)r2.z | ((uint64_t)(uint32_t)r2.w << 32);
                    if (better(r2.x, g2, ck, cg, lo, hi)) {
                        ck = r2.x;
                        cg = g2;
                    }
                }
                warp_best(ck, cg, lo, hi);
                if (!LEARNED || kind == kPlain) {
                    finish_segment(P, d, it.series, lo, hi, ck, cg, epoch);
                } else if (kind == kRefine) {
                    const CertRecord *rec = P.recs + it.rec;
                    const int rk = __ldcg(&rec->best_k);
                    const uint64_t rg = __ldcg(&rec->best_g);
                    if (better(rk, rg, ck, cg, lo, hi)) {
                        ck = rk;
                        cg = rg;
                    }
                    finish_segment(P, d, it.series, lo, hi, ck, cg, epoch);
                } else {
                    certify_segment(P, d, it, ck, cg, epoch);
                }
            }
        }
        if (lane == 0) {
            __threadfence();
            atomicAdd((unsigned long long *)&P.q->pending, (unsigned long long)(-1ll));
        }
        __syncwarp();
    }
    if (lane == 0 && my_evals) atomicAdd(&P.q->evals, my_evals);
    if (lane == 0 && my_swept) atomicAdd(&P.q->swept, my_swept);
}

// Expand the top-level slices of every series into the queue, costliest series first.
__global__ void init_items_kernel(const SeriesDesc *__restrict__ desc, const int32_t *__restrict__ qorder,
                                  const int64_t *__restrict__ item_base, int64_t S, int32_t min_seg,
                                  int32_t top_parts, WorkItem *items, int32_t *ready, uint32_t *gcount,
                                  uint32_t epoch) {
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= S) return;
    const int32_t s = qorder[i];
    const int32_t T = desc[s].T;
    const bool sweep = desc[s].kpt == 0;
    const int nch = sweep ? sweep_parts(T, min_seg, top_parts) : seg_chunks(T, min_seg, desc[s].kpt);
    const int64_t b = item_base[i];
    for (int c = lane; c < nch; c += 32) {
        int k0 = 0, k1 = T - min_seg;
        if (sweep) sweep_part_range(min_seg, T - min_seg, c, nch, k0, k1);
        int4 *dst = reinterpret_cast<int4 *>(items + b + c);
        dst[0] = make_int4(s, 0, T, c);
        dst[1] = make_int4(kPlain | (nch << 8), k0, k1, sweep ? kSweepItem : -1);
        if (c == 0) gcount[b] = 0;
        ready[b + c] = (int32_t)epoch;
    }
}

// Learned segmentation: decide each series' path from its proposal confidence (plain scan
// when conf < conf_min, or when the run sweep takes the series) and push the work for its
// whole range.
__global__ void init_learned_kernel(RunParams P, const float *__restrict__ conf, float conf_min,
                                    int32_t *__restrict__ fallback_out, int64_t S, uint32_t epoch) {
    const int64_t s = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (s >= S) return;
    const SeriesDesc d = P.desc[s];
    // the run sweep's cost per split is below the probes': series it takes are scanned in full
    const bool swept = P.rk != nullptr && d.kpt == 0 && d.nruns <= kSweepMaxRuns;
    if (lane == 0) fallback_out[s] = (conf[s] < conf_min || (swept && !P.win_only)) ? 1 : 0;
    __syncwarp();
    __threadfence_block();
    push_segment(P, d, (int)s, 0, d.T, epoch, P.top_parts);
}

// One warp per series: gather the flagged steps in ascending order.
__global__ void collect_kernel(const SeriesDesc *__restrict__ desc, int64_t S, const uint8_t *__restrict__ cp_flag,
                               const int64_t *__restrict__ cp_num, const int64_t *__restrict__ cp_den,
                               const double *__restrict__ cp_p, const double *__restrict__ cp_crit, int32_t max_cp,
                               int32_t *cp_count, int32_t *cp_idx, int64_t *dnum, int64_t *dden, double *p,
                               double *crit, QueueHeader *q) {
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
                if (crit) crit[o] = cp_crit[d.step_base + t];
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
        if (crit) crit[o] = 0.0;
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
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, queue_kernel<true, false>, kScanThreads, 0) !=
        cudaSuccess)
        return 0;
    return sms * (per_sm > 0 ? per_sm : 1);
}

int queue_grid_sweep(int device) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    // one grid for every sweep instantiation: the smallest residency among them
    int per[5] = {0, 0, 0, 0, 0};
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[0], queue_kernel<false, true>, kSweepThreads, 0) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[1], queue_kernel<true, true>, kSweepThreads, 0) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[2], queue_kernel<false, true, kWalkSkip>, kSweepThreads,
                                                      0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[3], queue_kernel<true, true, kWalkSkip>, kSweepThreads,
                                                      0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[4], queue_kernel<true, true, kWalkWindows>, kSweepThreads,
                                                      0) != cudaSuccess)
        return 0;
    int per_sm = per[0];
    for (int i = 1; i < 5; i++) per_sm = std::min(per_sm, per[i]);
    return sms * (per_sm > 0 ? per_sm : 1);
}

cudaError_t launch_queue_run(const RunParams &P, int grid, uint32_t epoch, cudaStream_t st) {
    if (P.mode == kRunLearned && P.rk && P.win_only)
        queue_kernel<true, true, kWalkWindows><<<grid, kSweepThreads, 0, st>>>(P, epoch);
    else if (P.mode == kRunLearned && P.rk) {
        // A learned call whose every series the sweep takes has no learned work left (each series
        // falls back to the full scan, and push_segment then pushes plain items only), so the
        // plain instantiation, lighter by the learned routing, gives the same answers.  Both are
        // launched; each reads the sort's count of unswept series first, and one of them works.
        RunParams Pa = P, Pl = P;
        Pa.gate = kGateAllSwept;
        Pl.gate = kGateSomeUnswept;
        if (P.sweep_skip) {
            queue_kernel<false, true, kWalkSkip><<<grid, kSweepThreads, 0, st>>>(Pa, epoch);
            queue_kernel<true, true, kWalkSkip><<<grid, kSweepThreads, 0, st>>>(Pl, epoch);
        } else {
            queue_kernel<false, true><<<grid, kSweepThreads, 0, st>>>(Pa, epoch);
            queue_kernel<true, true><<<grid, kSweepThreads, 0, st>>>(Pl, epoch);
        }
    }
    else if (P.mode == kRunLearned)
        queue_kernel<true, false><<<grid, kScanThreads, 0, st>>>(P, epoch);
    else if (P.rk && P.sweep_skip)
        queue_kernel<false, true, kWalkSkip><<<grid, kSweepThreads, 0, st>>>(P, epoch);
    else if (P.rk)
        queue_kernel<false, true><<<grid, kSweepThreads, 0, st>>>(P, epoch);
    else
        queue_kernel<false, false><<<grid, kScanThreads, 0, st>>>(P, epoch);
    return cudaGetLastError();
}

cudaError_t launch_init_learned(const RunParams &P, const float *conf, float conf_min, int32_t *fallback_out,
                                int64_t S, uint32_t epoch, cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    const int warps = 8;
    init_learned_kernel<<<(unsigned)((S + warps - 1) / warps), warps * 32, 0, st>>>(P, conf, conf_min, fallback_out, S,
                                                                                      epoch);
    return cudaGetLastError();
}

cudaError_t launch_init_items(const SeriesDesc *desc, const int32_t *qorder, const int64_t *item_base, int64_t S,
                              int32_t min_seg, int32_t top_parts, WorkItem *items, int32_t *ready, uint32_t *gcount,
                              uint32_t epoch, cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    const int warps = 8;
    init_items_kernel<<<(unsigned)((S + warps - 1) / warps), warps * 32, 0, st>>>(
        desc, qorder, item_base, S, min_seg, top_parts, items, ready, gcount, epoch);
    return cudaGetLastError();
}

cudaError_t launch_collect(const SeriesDesc *desc, int64_t S, const uint8_t *cp_flag, const int64_t *cp_num,
                           const int64_t *cp_den, const double *cp_p, const double *cp_crit, int32_t max_cp,
                           int32_t *cp_count, int32_t *cp_idx, int64_t *dnum, int64_t *dden, double *p, double *crit,
                           QueueHeader *q, cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    const int warps = 8;
    const unsigned blocks = (unsigned)((S + warps - 1) / warps);
    collect_kernel<<<blocks, warps * 32, 0, st>>>(desc, S, cp_flag, cp_num, cp_den, cp_p, cp_crit, max_cp, cp_count,
                                                  cp_idx, dnum, dden, p, crit, q);
    return cudaGetLastError();
}

}  // namespace mt4g
