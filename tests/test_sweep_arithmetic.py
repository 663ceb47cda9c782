"""CPU checks of the arithmetic the run sweep and the counting sort are built on.

The CUDA kernels cannot run here; these tests replay, in plain Python integers reduced to 32 bits
the way the kernels' registers wrap, the formulation the kernels use, and compare it with the
definition g_k = max_x |H c_L(x) - a C(x)| (Sec. II-C-1, Sec. IV-B-1 (4)) evaluated by brute force.
What is pinned:
  - the per-lane blocks of runs: R = ceil(U'/32) rounded up to a multiple of 8 (at least 8), the
    same for all 32 lanes, positions at or past U' padded with l = 0 and C = N,
  - the padded layout (lane stride R + 4 words) and the run -> layout position map, within
    the stage's 32 (48 + 4) words, and the evaluation's loads two quads ahead within its tail,
  - values accumulated relative to the run before each block, four runs per 16-byte load, with the
    block's offset taken from a scan of the blocks' sums of l afterwards,
  - the counting sort's run table, run indices and nearest-rank order statistics.
The GPU parity tests (-m gpu) compare the kernels themselves with the oracle.
"""
import numpy as np
import pytest

M32 = 1 << 32


def s32(v):
    v %= M32
    return v - M32 if v >= 1 << 31 else v


def brute_g(x, m, lo, hi):
    seg = np.sort(x[lo * m:hi * m])
    vals = np.unique(seg)
    C = np.searchsorted(seg, vals, side="right").astype(np.int64)
    H = hi - lo
    out = {}
    for k in range(lo + 1, hi):
        cl = np.searchsorted(np.sort(x[lo * m:k * m]), vals, side="right").astype(np.int64)
        out[k] = int(np.max(np.abs(H * cl - (k - lo) * C)))
    return out


MAX_R, STAGE_WORDS, STAGE_TAIL = 48, 32 * (48 + 4), 16


def lane_blocks(Uc):
    """Block size R, lane stride Rs and each lane's first run."""
    R = max(8, -(-((Uc + 31) // 32) // 8) * 8)
    Rs = R + 4
    return R, Rs, [L * R for L in range(32)]


def sweep_g(x, m, lo, hi, A, B):
    """The sweep's arithmetic: compact runs, padded lane blocks, relative values, block-sum scan."""
    dv = np.unique(x)
    rk = np.searchsorted(dv, x)
    H = hi - lo
    cnt = np.bincount(rk[lo * m:hi * m], minlength=len(dv))
    keep = np.nonzero(cnt)[0]
    Uc = len(keep)
    R, Rs, firsts = lane_blocks(Uc)
    assert R <= MAX_R and 32 * Rs <= STAGE_WORDS
    pos = np.full(len(dv), -1)
    pos[keep] = [(ci // R) * Rs + ci % R for ci in range(Uc)]
    assert pos.max() < 32 * Rs and len(set(pos[keep].tolist())) == Uc
    C = [int(c) % M32 for c in np.cumsum(cnt[keep])]
    N = C[-1]
    assert N == m * H
    l = [0] * (32 * Rs)

    def add_step(t):
        for j in range(m):
            c = pos[rk[t * m + j]]
            l[c] = (l[c] + H) % M32

    for t in range(lo, A):
        add_step(t)
    res = {}
    for k in range(A, B + 1):
        a = k - lo
        sums, ext = [], []
        for L, b0 in enumerate(firsts):
            Cb = 0 if b0 == 0 else (C[b0 - 1] if b0 <= Uc else N)
            Cr = [C[b0 + j] if b0 + j < Uc else N for j in range(R)]
            h0 = (a * Cb) % M32
            hc, mx, mn = h0, -(1 << 31), (1 << 31) - 1
            for q in range(R // 4):  # one 16-byte load: four runs
                for j in range(4 * q, 4 * q + 4):
                    hc = (hc + l[L * Rs + j]) % M32
                    v = s32(hc + (M32 - a) * Cr[j])
                    mx, mn = max(mx, v), min(mn, v)
            sums.append((hc - h0) % M32)
            ext.append((Cb, mx, mn))
        carry, g = 0, 0
        for blk, (Cb, mx, mn) in zip(sums, ext):
            vs = (carry - a * Cb) % M32
            g = max(g, s32(vs + mx % M32), -s32(vs + mn % M32), 0)
            carry = (carry + blk) % M32
        res[k] = g
        if k < B:
            add_step(k)
    return res


@pytest.mark.parametrize("seed", range(6))
def test_sweep_arithmetic_matches_definition(seed):
    rng = np.random.default_rng(100 + seed)
    for _ in range(8):
        T = int(rng.integers(4, 40))
        m = int(rng.integers(1, 9))
        x = rng.integers(0, int(rng.integers(1, 2500)), size=T * m).astype(np.int64)
        x[int(rng.integers(0, T)) * m:] += int(rng.integers(0, 60))
        lo = int(rng.integers(0, T - 2))
        hi = int(rng.integers(lo + 2, T + 1))
        ms = int(rng.integers(1, max(2, (hi - lo) // 2 + 1)))
        A, B = lo + ms, hi - ms
        if B < A:
            continue
        assert m * (hi - lo) ** 2 < 1 << 31
        bf, sw = brute_g(x, m, lo, hi), sweep_g(x, m, lo, hi, A, B)
        assert all(bf[k] == sw[k] for k in range(A, B + 1))


def test_lane_blocks_cover_every_size():
    """For every U' up to the sweep's 1536 runs: 32 blocks of R runs cover [0, U'), R <= 48 is a
    multiple of 8, the layout fits the stage, the evaluation's loads (groups of two quads, the next
    group loaded before the current one is evaluated) stay within the stage and its tail, and the
    eight lanes of a quarter warp start their 16-byte loads on eight different four-bank groups
    (lane stride Rs = 4 mod 8)."""
    for Uc in range(1, 1537):
        R, Rs, firsts = lane_blocks(Uc)
        assert R % 8 == 0 and 8 <= R <= MAX_R and 32 * R >= Uc and 32 * Rs <= STAGE_WORDS
        assert R == 8 or 32 * (R - 8) < Uc  # no larger than needed
        magic = 65536 // (R // 8) + 1  # the kernel's layout position ci + 4 floor(ci / R)
        assert all(ci + 4 * (((ci >> 3) * magic) >> 16) == (ci // R) * Rs + ci % R for ci in range(Uc))
        nq = R // 4
        last_quad = max(2 * g + 3 for g in range(nq // 2))  # quads 0 and 1 first, then 2g+2, 2g+3
        assert 31 * Rs + 4 * last_quad + 3 < STAGE_WORDS + STAGE_TAIL
        assert Rs % 8 == 4
        for q in range(R // 4):
            for L0 in range(0, 32, 8):
                groups = {((L * Rs + 4 * q) // 4) % 8 for L in range(L0, L0 + 8)}
                assert len(groups) == 8


def test_counting_sort_tables():
    """Counting path: value counts -> run table, run indices and the nearest-rank statistics
    (sorted value at N/2 and at ceil(qN) - 1 for q = 1/2, 95/100)."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        N = int(rng.integers(2, 5000))
        vmin = int(rng.integers(0, 1 << 31))
        x = vmin + rng.integers(0, int(rng.integers(1, 3000)), size=N)
        span = int(x.max() - x.min() + 1)
        cnt = np.bincount(x - x.min(), minlength=span)
        present = np.nonzero(cnt)[0]
        rt = np.concatenate([[0], np.cumsum(cnt[present])])
        rank = np.zeros(span, np.int64)
        rank[present] = np.arange(len(present))
        ranks = rank[x - x.min()]
        s = np.sort(x)
        assert np.array_equal(np.unique(x)[ranks], x)
        assert np.array_equal(rt[:-1], np.searchsorted(s, np.unique(x)))
        for q in (N // 2, (50 * N + 99) // 100 - 1, (95 * N + 99) // 100 - 1):
            r = int(np.searchsorted(rt, q, side="right") - 1)
            assert x.min() + present[r] == s[q]

