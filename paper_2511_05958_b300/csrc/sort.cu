// Per-series LSD radix sort of the latency samples, carrying step labels, and
// the run table of distinct values.
//
// The ECDFs of Sec. II-C-1 are read off the pooled samples in value order, so each
// series is sorted once: ascending by value, equal values in step order (the input
// is step-major and every pass is stable).  One CTA owns one series and runs all of
// its 8-bit digit passes itself, as many as the series' largest value needs.  When
// every value is below 2^16 the key is (value << 16) | step, so a pass moves 4 bytes
// per sample; otherwise values and 16-bit labels move separately.  The first read
// also counts the first digit, and each pass counts the next one while it ranks.
//
// Within a 2048-sample tile, each warp ranks its 256 samples by digit-peer masks
// (stable: item-major, then lane order), per-warp digit counts are scanned across warps, the tile is staged in shared memory in sorted order and written out so
// that consecutive positions of a digit go to consecutive addresses; a running
// per-digit base carries the order across tiles.  The last step writes the labels
// in value order to labA and the start of every run of equal values.  For series with at
// most kSweepMaxRuns distinct values a final read writes every sample's run index, in input
// order, to labB (the scan's run sweep reads it step by step).
#include <type_traits>

#include "mt4g_internal.cuh"

namespace mt4g {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// L2 eviction priorities for the counting path (createpolicy + L2::cache_hint operands): the
// samples are read once (evict first), the 2-byte table offsets written by the first read must
// survive until the second pass reads them back (evict last), and the final run indices are not
// read again by this kernel (evict first).
__device__ __forceinline__ uint64_t pol_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t pol_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint4 ld_hint(const uint4 *a, uint64_t pol) {
    uint4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_hint(uint2 *a, uint2 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.u32 [%0], {%1,%2}, %3;" ::"l"(a), "r"(v.x), "r"(v.y), "l"(pol) : "memory");
}
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

// Exclusive scan of s_in[0..255] into s_out[0..255] by the first 256 threads.
// Must be called by all threads of the block (contains __syncthreads).
__device__ void scan256(const uint32_t *s_in, uint32_t *s_out, uint32_t *s_tmp) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t v = 0, incl = 0;
    if (tid < 256) {
        v = s_in[tid];
        incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_tmp[warp] = incl;
    }
    __syncthreads();
    if (tid < 256) {
        uint32_t wbase = 0;
        for (int w = 0; w < warp; w++) wbase += s_tmp[w];
        s_out[tid] = wbase + incl - v;
    }
    __syncthreads();
}

// Lanes of vm holding the same 8-bit digit as this lane (every lane of the warp must call it):
// one match.any.  A choice by the warp's digit range between match.any and eight ballots, with
// two reductions to make it, was slower on B300 (uneven workload sort 44.9 against 42.1 ms;
// eight ballots alone 53.0 ms).
__device__ __forceinline__ unsigned digit_peers(uint32_t dg, unsigned vm) { return __match_any_sync(kFull, dg) & vm; }

// Shared-memory histogram increment (lanes outside vm add nothing): a plain atomic per lane.
// The hardware resolves lanes that hit the same counter; aggregating them per warp first (two
// reductions and a match.any) cost more on B300, even for the all-equal high digits of a series
// (uneven workload sort 51.7 ms that way, 44.7 ms this way).
__device__ __forceinline__ void hist_add(uint32_t *h, uint32_t dg, unsigned vm) {
    if ((vm >> (threadIdx.x & 31)) & 1u) atomicAdd(h + dg, 1u);
}

// e / m for 0 <= e < 2^30 by a single-precision reciprocal and an exact correction.
__device__ __forceinline__ uint32_t div_step(uint32_t e, uint32_t m, float inv_m) {
    uint32_t t = __float2uint_rz((float)e * inv_m);
    const uint32_t r = t * m;
    if (r > e) t -= (r - e + m - 1) / m;                // at most a couple of steps
    else if (e - r >= m) t += (e - r) / m;
    return t;
}

constexpr int kCountWords = 11552;  // the counting table (46 KB; four CTAs per SM)
constexpr int kSortFieldWords = kSortWarps * 256 + 5 * 256 + kSortTile + kSortTile / 2 + 32;

struct SortSmem {
    uint32_t wc[kSortWarps][256];  // per-warp digit counts -> tile-local offsets
    uint32_t hist[256];            // digit counts of the current pass (whole series)
    uint32_t hist2[256];           // digit counts of the next pass
    uint32_t base[256];            // global start of each digit before the current tile
    uint32_t tstart[256];          // tile-local start of each digit
    uint32_t tcnt[256];            // tile digit counts
    uint32_t key[kSortTile];       // tile staged in sorted order
    uint16_t lab[kSortTile];
    uint32_t tmp[32];
    // the counting path uses the whole struct as kFastSpan 32-bit counters
    uint32_t spare[kCountWords > kSortFieldWords ? kCountWords - kSortFieldWords : 1];
};

// LSD passes over one series.  COMP: keys are (value << 16) | step (value < 2^16), the
// step label rides in the low half; otherwise keys are the values and labels travel in
// their own arrays.  Pass p uses value bits [8p, 8p + 8).  Pass p reads (p == 0: the
// input; odd p: B; even p: A) and writes the other buffer.  On entry sm.hist holds the
// digit counts of pass 0.
template <bool COMP>
__device__ void lsd_passes(SortSmem &sm, int passes, const uint32_t *__restrict__ in, int32_t N, int32_t m,
                           uint32_t *keyA, uint32_t *keyB, uint16_t *labA, uint16_t *labB) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float inv_m = 1.0f / (float)m;
    for (int p = 0; p < passes; p++) {
        const int shift = 8 * p;
        const uint32_t *src_key = (p & 1) ? keyB : keyA;
        const uint16_t *src_lab = (p & 1) ? labB : labA;
        uint32_t *dst_key = (p & 1) ? keyA : keyB;
        uint16_t *dst_lab = (p & 1) ? labA : labB;
        const bool has_next = p + 1 < passes;
        scan256(sm.hist, sm.base, sm.tmp);
        if (tid < 256) sm.hist2[tid] = 0;
        __syncthreads();
        // one tile; FULL: the tile lies wholly inside the series (every tile but the last), so
        // no sample is tested against N
        auto tile = [&](const int tb, auto full_c) {
            constexpr bool FULL = decltype(full_c)::value;
            const int tn = FULL ? kSortTile : min(kSortTile, N - tb);
            for (int j = lane; j < 256; j += 32) sm.wc[warp][j] = 0;
            __syncwarp();
            uint32_t key[kSortItems], rk[kSortItems];
            uint16_t lb[kSortItems];
            // all loads of the tile first, so they are in flight together
#pragma unroll
            for (int it = 0; it < kSortItems; it++) {
                const int e = tb + warp * (32 * kSortItems) + it * 32 + lane;
                key[it] = 0;
                lb[it] = 0;
                if (FULL || e < N) {
                    if (p == 0) {
                        key[it] = __ldg(in + e);
                    } else {
                        key[it] = src_key[e];
                        if (!COMP) lb[it] = src_lab[e];
                    }
                }
            }
            if (p == 0) {
                // step label = sample index / m (a shift when m is a power of two, as it usually is)
                const bool pow2 = (m & (m - 1)) == 0;
                const int msh = __ffs(m) - 1;
#pragma unroll
                for (int it = 0; it < kSortItems; it++) {
                    const int e = tb + warp * (32 * kSortItems) + it * 32 + lane;
                    const uint32_t ec = FULL ? (uint32_t)e : (uint32_t)min(e, N - 1);
                    const uint32_t t = pow2 ? ec >> msh : div_step(ec, (uint32_t)m, inv_m);
                    if (COMP) key[it] = (key[it] << 16) | t;
                    lb[it] = (uint16_t)t;
                }
            }
#pragma unroll
            for (int it = 0; it < kSortItems; it++) {
                const int e = tb + warp * (32 * kSortItems) + it * 32 + lane;
                const bool valid = FULL || e < N;
                const unsigned vm = FULL ? kFull : __ballot_sync(kFull, valid);
                const uint32_t val = COMP ? key[it] >> 16 : key[it];
                const uint32_t dg = (val >> shift) & 255u;
                const unsigned peers = digit_peers(dg, vm);
                const int leader = valid ? __ffs(peers) - 1 : 0;
                uint32_t old = 0;
                if (valid && lane == leader) {
                    old = sm.wc[warp][dg];
                    sm.wc[warp][dg] = old + (uint32_t)__popc(peers);
                }
                old = __shfl_sync(kFull, old, leader);
                rk[it] = old + (uint32_t)__popc(peers & lanemask_lt());
                if (has_next) hist_add(sm.hist2, (val >> (shift + 8)) & 255u, vm);
                __syncwarp();
            }
            __syncthreads();
            if (tid < 256) {
                uint32_t tot = 0;
#pragma unroll
                for (int w = 0; w < kSortWarps; w++) tot += sm.wc[w][tid];
                sm.tcnt[tid] = tot;
            }
            __syncthreads();
            scan256(sm.tcnt, sm.tstart, sm.tmp);
            if (tid < 256) {
                uint32_t run = sm.tstart[tid];
#pragma unroll
                for (int w = 0; w < kSortWarps; w++) {
                    const uint32_t c = sm.wc[w][tid];
                    sm.wc[w][tid] = run;
                    run += c;
                }
            }
            __syncthreads();
            // stage the tile in shared memory in sorted order
#pragma unroll
            for (int it = 0; it < kSortItems; it++) {
                const int e = tb + warp * (32 * kSortItems) + it * 32 + lane;
                if (FULL || e < N) {
                    const uint32_t val = COMP ? key[it] >> 16 : key[it];
                    const uint32_t dg = (val >> shift) & 255u;
                    const uint32_t local = sm.wc[warp][dg] + rk[it];
                    sm.key[local] = key[it];
                    if (!COMP) sm.lab[local] = lb[it];
                }
            }
            __syncthreads();
            // write out: consecutive tile positions of one digit go to consecutive addresses
            for (int i = tid; i < tn; i += kSortThreads) {
                const uint32_t k2 = sm.key[i];
                const uint32_t dg = ((COMP ? k2 >> 16 : k2) >> shift) & 255u;
                const uint32_t g = sm.base[dg] + (uint32_t)i - sm.tstart[dg];
                dst_key[g] = k2;
                if (!COMP) dst_lab[g] = sm.lab[i];
            }
            __syncthreads();
            if (tid < 256) sm.base[tid] += sm.tcnt[tid];
            __syncthreads();
        };
        for (int tb = 0; tb < N; tb += kSortTile) {
            if (tb + kSortTile <= N)
                tile(tb, std::true_type{});
            else
                tile(tb, std::false_type{});
        }
        if (tid < 256) sm.hist[tid] = sm.hist2[tid];
        __syncthreads();
    }
}

// Values per series the counting path can index: the sort's shared memory as 32-bit counters.
constexpr uint32_t kFastSpan = (uint32_t)kCountWords;
static_assert(kFastSpan * sizeof(uint32_t) <= sizeof(SortSmem), "counting table fits the sort's shared memory");
// The counting table's base is guessed from the series' first sample, this far below it (a
// latency series usually starts at its smallest latencies); a value outside the table sends the
// series to a recount from its true minimum.
constexpr uint32_t kBaseBelow = 1024;
constexpr int kCountVec = 4;  // 16-byte loads in flight per thread

// A series' samples as a head of single samples up to the first 16-byte boundary, 16-byte
// chunks, and a tail of single samples.
struct VecSplit {
    int head, nvec;
};
__device__ __forceinline__ VecSplit vec_split(const uint32_t *in, int32_t N) {
    const int head = min(N, (int)(((16u - (uint32_t)((uintptr_t)in & 15u)) & 15u) >> 2));
    return VecSplit{head, (N - head) >> 2};
}

// Block-wide min and max (all threads call it; every thread gets the result).  Uses its own
// shared words, so the counting table, which spans all of SortSmem, stays intact.
__device__ __forceinline__ void block_minmax(uint32_t &vmin, uint32_t &vmax) {
    __shared__ uint32_t s_mm[2][kSortWarps + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    vmax = __reduce_max_sync(kFull, vmax);
    vmin = __reduce_min_sync(kFull, vmin);
    __syncthreads();  // the previous call's results may still be read
    if (lane == 0) {
        s_mm[0][warp] = vmax;
        s_mm[1][warp] = vmin;
    }
    __syncthreads();
    if (warp == 0) {
        uint32_t v = lane < kSortWarps ? s_mm[0][lane] : 0u;
        uint32_t u = lane < kSortWarps ? s_mm[1][lane] : 0xffffffffu;
        v = __reduce_max_sync(kFull, v);
        u = __reduce_min_sync(kFull, u);
        if (lane == 0) {
            s_mm[0][kSortWarps] = v;
            s_mm[1][kSortWarps] = u;
        }
    }
    __syncthreads();
    vmax = s_mm[0][kSortWarps];
    vmin = s_mm[1][kSortWarps];
}

// One value into the counting table (every lane calls it; lanes with valid = false add nothing).
// A value outside [base, base + kFastSpan) is not counted and sets `out`.
__device__ __forceinline__ void count_one(uint32_t *cnt, uint32_t v, uint32_t base, bool valid, bool &out,
                                          uint32_t &vmin, uint32_t &vmax) {
    const uint32_t dv = v - base;
    const bool in_range = dv < kFastSpan;
    out |= valid && !in_range;
    if (valid) {
        vmin = min(vmin, v);
        vmax = max(vmax, v);
    }
    // a plain shared-memory atomic per sample: the hardware resolves lanes that hit the same
    // counter, which costs less here than aggregating them per warp first (two reductions and a
    // match.any per sample: the counting sort took 7.51 ms on c5 that way, 5.70 ms this way)
    if (valid && in_range) atomicAdd(cnt + dv, 1u);
}

// Count every sample's value - base into the table (the sort's shared memory as kFastSpan
// counters), reading the series once with 16-byte loads; also the series' min and max.  Each
// sample's table offset value - base (below kFastSpan, so 16 bits) goes to rko, in input order:
// the run indices are later written over it in place, and while the series is being counted
// these 2 bytes per sample stay in L2, unlike a second read of its 4-byte samples.  Returns
// false (the same in every thread) when some value fell outside the table (rko then holds
// nothing of use).
__device__ bool count_values(SortSmem &sm, const uint32_t *__restrict__ in, int32_t N, uint32_t base,
                             uint32_t &vmin, uint32_t &vmax, uint16_t *__restrict__ rko) {
    const int tid = threadIdx.x;
    uint32_t *cnt = reinterpret_cast<uint32_t *>(&sm);
    for (uint32_t i = tid; i < kFastSpan; i += kSortThreads) cnt[i] = 0;
    __syncthreads();
    const VecSplit vs = vec_split(in, N);
    vmin = 0xffffffffu;
    vmax = 0;
    bool out = false;
    {  // head and tail samples, one per thread of the first warp
        const int nt = N - vs.head - 4 * vs.nvec;
        if (tid < 32) {
            const int i = tid < vs.head ? tid : (tid - vs.head < nt ? vs.head + 4 * vs.nvec + (tid - vs.head) : -1);
            const uint32_t v = i >= 0 ? __ldg(in + i) : 0u;
            count_one(cnt, v, base, i >= 0, out, vmin, vmax);
            if (i >= 0) rko[i] = (uint16_t)(v - base);
        }
    }
    const uint4 *v4 = reinterpret_cast<const uint4 *>(in + vs.head);
    // rko + head is 8-byte aligned when the samples start on a 16-byte boundary (then off + head
    // is a multiple of 4 samples, and the label arrays are 256-byte aligned); else 2-byte stores
    uint16_t *o = rko + vs.head;
    const bool st8 = ((uintptr_t)o & 7u) == 0;  // the same for every thread
    int b0 = 0;
    if (st8) {  // whole rounds: no per-sample tests
        for (; b0 + kSortThreads * kCountVec <= vs.nvec; b0 += kSortThreads * kCountVec) {
            uint4 x[kCountVec];
#pragma unroll
            for (int it = 0; it < kCountVec; it++) x[it] = ld_hint(v4 + b0 + it * kSortThreads + tid, pol_first());
#pragma unroll
            for (int it = 0; it < kCountVec; it++) {
                count_one(cnt, x[it].x, base, true, out, vmin, vmax);
                count_one(cnt, x[it].y, base, true, out, vmin, vmax);
                count_one(cnt, x[it].z, base, true, out, vmin, vmax);
                count_one(cnt, x[it].w, base, true, out, vmin, vmax);
                st_hint(reinterpret_cast<uint2 *>(o) + b0 + it * kSortThreads + tid,
                        make_uint2(((x[it].x - base) & 0xffffu) | ((x[it].y - base) << 16),
                                   ((x[it].z - base) & 0xffffu) | ((x[it].w - base) << 16)), pol_last());
            }
        }
    }
    for (; b0 < vs.nvec; b0 += kSortThreads * kCountVec) {
        uint4 x[kCountVec];
#pragma unroll
        for (int it = 0; it < kCountVec; it++) {
            const int i = b0 + it * kSortThreads + tid;
            x[it] = i < vs.nvec ? ld_hint(v4 + i, pol_first()) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int it = 0; it < kCountVec; it++) {
            const bool valid = b0 + it * kSortThreads + tid < vs.nvec;
            count_one(cnt, x[it].x, base, valid, out, vmin, vmax);
            count_one(cnt, x[it].y, base, valid, out, vmin, vmax);
            count_one(cnt, x[it].z, base, valid, out, vmin, vmax);
            count_one(cnt, x[it].w, base, valid, out, vmin, vmax);
            if (valid) {
                const int i = b0 + it * kSortThreads + tid;
                if (st8) {
                    st_hint(reinterpret_cast<uint2 *>(o) + i, make_uint2(((x[it].x - base) & 0xffffu) | ((x[it].y - base) << 16),
                                                                 ((x[it].z - base) & 0xffffu) | ((x[it].w - base) << 16)), pol_last());
                } else {
                    o[4 * i] = (uint16_t)(x[it].x - base);
                    o[4 * i + 1] = (uint16_t)(x[it].y - base);
                    o[4 * i + 2] = (uint16_t)(x[it].z - base);
                    o[4 * i + 3] = (uint16_t)(x[it].w - base);
                }
            }
        }
    }
    out = __syncthreads_or(out);
    block_minmax(vmin, vmax);
    return !out;
}

// Counting path, after count_values succeeded: scans the table over [vmin, vmax] for the run
// table (starts of the distinct values in value order) and the order statistics, turns it into a
// value -> run index table, and writes each sample's run index in input order over the table
// offset count_values left there (8-byte reads and writes where aligned).  All threads call it;
// returns false, with nothing written, when the series has more than kSweepMaxRuns distinct
// values.  The sorted labels are not produced (kDescNoLabels).
__device__ bool count_runs(SortSmem &sm, const uint32_t *__restrict__ in, int32_t N, uint32_t base, uint32_t vmin,
                           uint32_t vmax, int32_t *__restrict__ rt, SeriesDesc *__restrict__ ds,
                           uint16_t *rko, unsigned long long *sweep_stats) {
    __shared__ uint32_t s_scan[2][kSortWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t *cnt = reinterpret_cast<uint32_t *>(&sm);
    const uint32_t t0 = vmin - base, span = vmax - vmin + 1;
    // each thread scans a contiguous piece of the table: distinct values and samples in it
    const uint32_t per = (span + kSortThreads - 1) / kSortThreads;
    const uint32_t c0 = t0 + min(span, (uint32_t)tid * per), c1 = t0 + min(span, (uint32_t)tid * per + per);
    uint32_t nd = 0, ns = 0;
    for (uint32_t i = c0; i < c1; i++) {
        const uint32_t c = cnt[i];
        nd += c != 0u;
        ns += c;
    }
    uint32_t id = nd, is = ns;  // inclusive warp scans
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, id, o), z = __shfl_up_sync(kFull, is, o);
        if (lane >= o) {
            id += y;
            is += z;
        }
    }
    if (lane == 31) {
        s_scan[0][warp] = id;
        s_scan[1][warp] = is;
    }
    __syncthreads();
    uint32_t bd = id - nd, bs = is - ns, U = 0;
    for (int w = 0; w < kSortWarps; w++) {
        const uint32_t a = s_scan[0][w], b = s_scan[1][w];
        if (w < warp) {
            bd += a;
            bs += b;
        }
        U += a;
    }
    if (U > (uint32_t)kSweepMaxRuns) return false;  // uniform: nothing written yet
    // run starts, order statistics (values at sorted positions N / 2 and ceil(q N) - 1), and
    // the value -> run index table in place of the counts
    const uint32_t qmed = (uint32_t)(N / 2), q50 = (uint32_t)((50 * (int64_t)N + 99) / 100 - 1),
                   q95 = (uint32_t)((95 * (int64_t)N + 99) / 100 - 1);
    uint32_t r = bd, pos = bs;
    for (uint32_t i = c0; i < c1; i++) {
        const uint32_t c = cnt[i];
        if (c == 0u) continue;
        rt[r] = (int32_t)pos;
        if (qmed - pos < c) ds->median = base + i;
        if (q50 - pos < c) ds->p50 = base + i;
        if (q95 - pos < c) ds->p95 = base + i;
        cnt[i] = r;
        r++;
        pos += c;
    }
    if (tid == 0) {
        rt[U] = N;
        ds->nruns = (int32_t)U;
        ds->flags |= kDescNoLabels;
        atomicAdd(sweep_stats, (unsigned long long)N);
        atomicAdd(sweep_stats + 1, (unsigned long long)N);
    }
    __syncthreads();
    // each sample's table offset (written in input order by count_values) becomes its run
    // index in place: coherent loads (the block wrote these words), 8 bytes = four samples
    const VecSplit vs = vec_split(in, N);
    if (tid < 32) {  // head and tail samples
        const int nt = N - vs.head - 4 * vs.nvec;
        const int i = tid < vs.head ? tid : (tid - vs.head < nt ? vs.head + 4 * vs.nvec + (tid - vs.head) : -1);
        if (i >= 0) rko[i] = (uint16_t)cnt[rko[i]];
    }
    uint16_t *o = rko + vs.head;
    if (((uintptr_t)o & 7u) == 0) {  // the same for every thread
        uint2 *o8 = reinterpret_cast<uint2 *>(o);
        int b0 = 0;
        for (; b0 + kSortThreads * 8 <= vs.nvec; b0 += kSortThreads * 8) {  // whole rounds: no tests
            uint2 x[8];
#pragma unroll
            for (int it = 0; it < 8; it++) x[it] = o8[b0 + it * kSortThreads + tid];
#pragma unroll
            for (int it = 0; it < 8; it++) {
                const uint32_t r0 = cnt[x[it].x & 0xffffu], r1 = cnt[x[it].x >> 16];
                const uint32_t r2 = cnt[x[it].y & 0xffffu], r3 = cnt[x[it].y >> 16];
                st_hint(o8 + b0 + it * kSortThreads + tid, make_uint2(r0 | (r1 << 16), r2 | (r3 << 16)), pol_first());
            }
        }
        for (; b0 < vs.nvec; b0 += kSortThreads * kCountVec) {
            uint2 x[kCountVec];
#pragma unroll
            for (int it = 0; it < kCountVec; it++) {
                const int i = b0 + it * kSortThreads + tid;
                x[it] = i < vs.nvec ? o8[i] : make_uint2(0u, 0u);
            }
#pragma unroll
            for (int it = 0; it < kCountVec; it++) {
                const int i = b0 + it * kSortThreads + tid;
                if (i < vs.nvec) {
                    const uint32_t r0 = cnt[x[it].x & 0xffffu], r1 = cnt[x[it].x >> 16];
                    const uint32_t r2 = cnt[x[it].y & 0xffffu], r3 = cnt[x[it].y >> 16];
                    st_hint(o8 + i, make_uint2(r0 | (r1 << 16), r2 | (r3 << 16)), pol_first());
                }
            }
        }
    } else {
        for (int i = tid; i < 4 * vs.nvec; i += kSortThreads) o[i] = (uint16_t)cnt[o[i]];
    }
    return true;
}

// Pass-0 digit counts and the min and max of the series in one read (16-byte loads).
__device__ void digit0_minmax(SortSmem &sm, const uint32_t *__restrict__ in, int32_t N, uint32_t &vmin,
                              uint32_t &vmax) {
    const int tid = threadIdx.x;
    if (tid < 256) sm.hist[tid] = 0;
    __syncthreads();
    vmin = 0xffffffffu;
    vmax = 0;
    const VecSplit vs = vec_split(in, N);
    if (tid < 32) {
        const int nt = N - vs.head - 4 * vs.nvec;
        const int i = tid < vs.head ? tid : (tid - vs.head < nt ? vs.head + 4 * vs.nvec + (tid - vs.head) : -1);
        const uint32_t v = i >= 0 ? __ldg(in + i) : 0u;
        if (i >= 0) {
            vmin = min(vmin, v);
            vmax = max(vmax, v);
        }
        hist_add(sm.hist, v & 255u, __ballot_sync(kFull, i >= 0));
    }
    const uint4 *v4 = reinterpret_cast<const uint4 *>(in + vs.head);
    for (int b0 = 0; b0 < vs.nvec; b0 += kSortThreads * kCountVec) {
        uint4 x[kCountVec];
#pragma unroll
        for (int it = 0; it < kCountVec; it++) {
            const int i = b0 + it * kSortThreads + tid;
            x[it] = i < vs.nvec ? __ldg(v4 + i) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int it = 0; it < kCountVec; it++) {
            const bool valid = b0 + it * kSortThreads + tid < vs.nvec;
            const unsigned vm = __ballot_sync(kFull, valid);
            if (valid) {
                vmin = min(min(vmin, x[it].x), min(x[it].y, min(x[it].z, x[it].w)));
                vmax = max(max(vmax, x[it].x), max(x[it].y, max(x[it].z, x[it].w)));
            }
            hist_add(sm.hist, x[it].x & 255u, vm);
            hist_add(sm.hist, x[it].y & 255u, vm);
            hist_add(sm.hist, x[it].z & 255u, vm);
            hist_add(sm.hist, x[it].w & 255u, vm);
        }
    }
    __syncthreads();
    block_minmax(vmin, vmax);
}

__global__ void __launch_bounds__(kSortThreads, 4)
sort_series_kernel(const uint32_t *__restrict__ samples, SeriesDesc *__restrict__ desc,
                   const int32_t *__restrict__ order, uint32_t *__restrict__ keyA, uint32_t *__restrict__ keyB,
                   uint16_t *__restrict__ labA, uint16_t *__restrict__ labB, int32_t *__restrict__ runs,
                   unsigned long long *sweep_stats) {
    __shared__ SortSmem sm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s = order[blockIdx.x];
    const SeriesDesc d = desc[s];
    const int64_t off = d.off;
    const int32_t m = d.m;
    const int32_t N = d.T * m;
    const uint32_t *in = samples + off;
    int32_t *rt = runs + d.run_base;
    uint32_t vmin, vmax;

    // ---- counting path: a run-sweep series with a narrow value span whose every segment the
    // sweep takes (m T^2 < 2^31) needs only the run table and the run indices.  One read counts
    // the values in a table based just below the first sample; if a value falls outside it and
    // the span still fits, a second read recounts from the minimum.
    if (sweep_stats && d.kpt == 0 && (uint64_t)m * (uint64_t)d.T * (uint64_t)d.T < (1ull << 31)) {
        const uint32_t v0 = __ldg(in);
        // the table [base, base + kFastSpan) must not wrap past 2^32 - 1
        uint32_t base = min(v0 - min(v0, kBaseBelow), 0xffffffffu - kFastSpan + 1u);
        bool ok = count_values(sm, in, N, base, vmin, vmax, labB + off);
        if (!ok && vmax - vmin < kFastSpan) {
            base = vmin;
            ok = count_values(sm, in, N, base, vmin, vmax, labB + off);
        }
        if (ok && count_runs(sm, in, N, base, vmin, vmax, rt, desc + s, labB + off, sweep_stats)) return;
        // too many distinct values (or too wide a span) for the counting path: radix sort
        __syncthreads();
    }
    digit0_minmax(sm, in, N, vmin, vmax);
    const int bits = vmax ? 32 - __clz(vmax) : 0;
    const int passes = max(1, (bits + 7) / 8);
    const bool comp = vmax < 65536u;
    uint32_t *kA = keyA + off, *kB = keyB + off;
    uint16_t *lA = labA + off, *lB = labB + off;
    if (comp)
        lsd_passes<true>(sm, passes, in, N, m, kA, kB, lA, lB);
    else
        lsd_passes<false>(sm, passes, in, N, m, kA, kB, lA, lB);

    // ---- run table and final labels (into labA), 8 consecutive samples per thread per round
    const uint32_t *fk = (passes & 1) ? kB : kA;
    const uint16_t *flab = (passes & 1) ? lB : lA;
    uint32_t count = 0;
    constexpr int kRunItems = 8;
    for (int tb = 0; tb < N; tb += kSortThreads * kRunItems) {
        const int i0 = tb + tid * kRunItems;
        uint32_t v[kRunItems + 1];
#pragma unroll
        for (int q = 0; q <= kRunItems; q++) {
            const int i = i0 + q - 1;
            const uint32_t k2 = (i >= 0 && i < N) ? fk[i] : 0u;
            v[q] = comp ? k2 >> 16 : k2;
            if (q > 0 && i < N) {
                if (comp)
                    lA[i] = (uint16_t)(k2 & 0xffffu);
                else if (passes & 1)
                    lA[i] = flab[i];
            }
        }
        uint32_t fl = 0;  // bit q: sample i0 + q starts a run
#pragma unroll
        for (int q = 0; q < kRunItems; q++) {
            const int i = i0 + q;
            if (i < N && (i == 0 || v[q + 1] != v[q])) fl |= 1u << q;
        }
        const uint32_t mine = (uint32_t)__popc(fl);
        uint32_t incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) sm.tmp[warp] = incl;
        __syncthreads();
        uint32_t before = 0, total = 0;
        if (lane < kSortWarps) {
            const uint32_t c = sm.tmp[lane];
            before = lane < warp ? c : 0;
            total = c;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            before += __shfl_xor_sync(kFull, before, o);
            total += __shfl_xor_sync(kFull, total, o);
        }
        uint32_t pos = count + before + incl - mine;
#pragma unroll
        for (int q = 0; q < kRunItems; q++)
            if (fl & (1u << q)) rt[pos++] = i0 + q;
        count += total;
        __syncthreads();
    }
    if (tid == 0) {
        rt[count] = N;
        desc[s].nruns = (int32_t)count;
        const uint32_t km = fk[N / 2];
        desc[s].median = comp ? km >> 16 : km;
        const uint32_t k50 = fk[(50 * (int64_t)N + 99) / 100 - 1], k95 = fk[(95 * (int64_t)N + 99) / 100 - 1];
        desc[s].p50 = comp ? k50 >> 16 : k50;
        desc[s].p95 = comp ? k95 >> 16 : k95;
    }

    // ---- run index of every sample in input order (labB), for the run sweep of the scan.
    // Runs are numbered in value order, so a sample's run index is its rank among the
    // series' distinct values: a table indexed by value when the value span fits in the
    // shared memory the passes no longer need, else a binary search over the distinct values.
    if (sweep_stats && tid == 0 && !(d.kpt == 0 && count <= (uint32_t)kSweepMaxRuns))
        atomicAdd(sweep_stats + 2, 1ull);  // a series the sweep does not take
    if (sweep_stats && count <= (uint32_t)kSweepMaxRuns) {
        if (tid == 0) atomicAdd(sweep_stats, (unsigned long long)N);
        constexpr uint32_t kLut = (uint32_t)(sizeof(SortSmem) / sizeof(uint16_t));
        uint16_t *lut = reinterpret_cast<uint16_t *>(&sm);
        uint32_t *dv = reinterpret_cast<uint32_t *>(&sm);
        const uint32_t kf = fk[0], kl = fk[N - 1];
        const uint32_t vmin = comp ? kf >> 16 : kf, vmax = comp ? kl >> 16 : kl;
        const bool use_lut = vmax - vmin < kLut;
        for (uint32_t r = tid; r < count; r += kSortThreads) {
            const uint32_t k2 = fk[rt[r]];
            const uint32_t v = comp ? k2 >> 16 : k2;
            if (use_lut)
                lut[v - vmin] = (uint16_t)r;
            else
                dv[r] = v;
        }
        __syncthreads();
        uint16_t *rko = labB + off;
        for (int b0 = 0; b0 < N; b0 += kSortThreads * kSortItems) {
            uint32_t v[kSortItems];
#pragma unroll
            for (int it = 0; it < kSortItems; it++) {
                const int i = b0 + it * kSortThreads + tid;
                v[it] = i < N ? __ldg(in + i) : vmin;
            }
#pragma unroll
            for (int it = 0; it < kSortItems; it++) {
                const int i = b0 + it * kSortThreads + tid;
                uint32_t r;
                if (use_lut) {
                    r = lut[v[it] - vmin];
                } else {
                    uint32_t a = 0, b = count - 1;
                    while (a < b) {
                        const uint32_t mid = (a + b) >> 1;
                        if (dv[mid] < v[it])
                            a = mid + 1;
                        else
                            b = mid;
                    }
                    r = a;
                }
                if (i < N) rko[i] = (uint16_t)r;
            }
        }
    }
}

// ---- Eq. 2 reduction (paper Sec. IV-B-1): S_t = sqrt(sum_j (r_tj - min r)^2), then
// each S_t replaced by its rank among the series' values (count of strictly smaller
// values).  Ranks preserve order and ties exactly, so the KS test on the ranks is
// the KS test on S.  The sum runs in j order with explicit round-to-nearest
// operations (no contraction into FMA).
__global__ void __launch_bounds__(256)
reduce_rank_kernel(const uint32_t *__restrict__ samples, const SeriesDesc *__restrict__ desc, double *red,
                   uint32_t *rank_out) {
    __shared__ uint32_t s_min[32];
    __shared__ double s_tile[1024];
    const int s = blockIdx.x;
    const SeriesDesc d = desc[s];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t N = (int64_t)d.T * d.m;
    const uint32_t *x = samples + d.off;
    uint32_t mn = 0xffffffffu;
    for (int64_t i = tid; i < N; i += blockDim.x) mn = min(mn, __ldg(x + i));
    mn = __reduce_min_sync(kFull, mn);
    if (lane == 0) s_min[warp] = mn;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = lane < (int)(blockDim.x / 32) ? s_min[lane] : 0xffffffffu;
        v = __reduce_min_sync(kFull, v);
        if (lane == 0) s_min[31] = v;
    }
    __syncthreads();
    mn = s_min[31];
    double *r = red + d.step_base;
    for (int t = tid; t < d.T; t += blockDim.x) {
        double acc = 0.0;
        const uint32_t *row = x + (int64_t)t * d.m;
        for (int j = 0; j < d.m; j++) {
            const double v = (double)(__ldg(row + j) - mn);
            acc = __dadd_rn(acc, __dmul_rn(v, v));
        }
        r[t] = __dsqrt_rn(acc);
    }
    __syncthreads();
    // ranks: number of strictly smaller reduced values
    for (int t0 = 0; t0 < d.T; t0 += blockDim.x) {
        const int t = t0 + tid;
        const double v = t < d.T ? r[t] : 0.0;
        uint32_t rank = 0;
        for (int u0 = 0; u0 < d.T; u0 += 1024) {
            __syncthreads();
            for (int u = tid; u < 1024; u += blockDim.x) s_tile[u] = (u0 + u < d.T) ? r[u0 + u] : 0.0;
            __syncthreads();
            const int nu = min(1024, d.T - u0);
            for (int u = 0; u < nu; u++) rank += s_tile[u] < v;
        }
        if (t < d.T) rank_out[d.step_base + t] = rank;
    }
}

// Invariants the scan relies on, checked per series (one CTA): the run table starts at 0,
// increases strictly and ends at N with nruns entries; every label is a step index (< T);
// labels are non-decreasing within each run (sample i and i - 1 in the same run, found by
// binary search in the validated table).  For kDescNoLabels series the labels are absent;
// instead every run index is below nruns and each run's count of them equals its length.
// Reads stay inside the series' label range [off, off + N) and run-table range
// [run_base, run_base + nruns].
__global__ void __launch_bounds__(256) check_sort_kernel(const SeriesDesc *__restrict__ desc,
                                                         const uint16_t *__restrict__ lab,
                                                         const uint16_t *__restrict__ rk,
                                                         const int32_t *__restrict__ runs, int32_t *status) {
    __shared__ uint32_t s_cnt[kSweepMaxRuns];
    const SeriesDesc d = desc[blockIdx.x];
    const int64_t N = (int64_t)d.T * d.m;
    const int32_t U = d.nruns;
    const int32_t *rt = runs + d.run_base;
    const bool nolab = (d.flags & kDescNoLabels) != 0;
    bool bad = U < 1 || U > N || (nolab && U > kSweepMaxRuns);
    if (!bad) {
        if (threadIdx.x == 0) bad = rt[0] != 0 || rt[U] != N;
        for (int32_t j = threadIdx.x; j < U && !bad; j += blockDim.x) bad = rt[j] >= rt[j + 1];
    }
    if (nolab) {
        const uint16_t *r = rk + d.off;
        for (int32_t j = threadIdx.x; j < kSweepMaxRuns; j += blockDim.x) s_cnt[j] = 0;
        __syncthreads();
        if (!__syncthreads_or(bad)) {
            for (int64_t i = threadIdx.x; i < N && !bad; i += blockDim.x) {
                const uint32_t v = r[i];
                if (v >= (uint32_t)U)
                    bad = true;
                else
                    atomicAdd(&s_cnt[v], 1u);
            }
            if (!__syncthreads_or(bad))
                for (int32_t j = threadIdx.x; j < U && !bad; j += blockDim.x) bad = s_cnt[j] != (uint32_t)(rt[j + 1] - rt[j]);
            bad = __syncthreads_or(bad);
        } else {
            bad = true;
        }
        if (bad && threadIdx.x == 0) atomicOr(status, (int32_t)kStatusCheck);
        return;
    }
    const uint16_t *l = lab + d.off;
    if (!bad)
        for (int64_t i = threadIdx.x; i < N && !bad; i += blockDim.x) bad = l[i] >= d.T;
    if (!__syncthreads_or(bad)) {
        for (int64_t i = 1 + threadIdx.x; i < N && !bad; i += blockDim.x) {
            int32_t lo = 0, hi = U;  // rt[lo] <= i < rt[hi]
            while (hi - lo > 1) {
                const int32_t mid = (lo + hi) >> 1;
                if (rt[mid] <= i)
                    lo = mid;
                else
                    hi = mid;
            }
            bad = rt[lo] != i && l[i - 1] > l[i];
        }
        bad = __syncthreads_or(bad);
    } else {
        bad = true;
    }
    if (bad && threadIdx.x == 0) atomicOr(status, (int32_t)kStatusCheck);
}

}  // namespace

cudaError_t launch_check_sort(const SeriesDesc *desc, int64_t S, const uint16_t *lab, const uint16_t *rk,
                              const int32_t *runs, int32_t *status, cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    check_sort_kernel<<<(unsigned)S, 256, 0, st>>>(desc, lab, rk, runs, status);
    return cudaGetLastError();
}

cudaError_t launch_sort(const uint32_t *samples, SeriesDesc *desc, const int32_t *order, int64_t S,
                        uint32_t *keyA, uint32_t *keyB, uint16_t *labA, uint16_t *labB, int32_t *runs,
                        unsigned long long *sweep_stats, cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    sort_series_kernel<<<(unsigned)S, kSortThreads, 0, st>>>(samples, desc, order, keyA, keyB, labA, labB, runs,
                                                             sweep_stats);
    return cudaGetLastError();
}

cudaError_t launch_reduce_rank(const uint32_t *samples, const SeriesDesc *raw_desc, int64_t S, double *red,
                               uint32_t *rank_out, cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    reduce_rank_kernel<<<(unsigned)S, 256, 0, st>>>(samples, raw_desc, red, rank_out);
    return cudaGetLastError();
}

}  // namespace mt4g
