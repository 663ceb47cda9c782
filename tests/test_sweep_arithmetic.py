"""CPU checks of the arithmetic the run sweep and the counting sort are built on.

The CUDA kernels cannot run here; these tests replay, in plain Python integers reduced to 32 bits
the way the kernels' registers wrap, the formulation the kernels use, and compare it with the
definition g_k = max_x |H c_L(x) - a C(x)| (Sec. II-C-1, Sec. IV-B-1 (4)) evaluated by brute force.
What is pinned:
  - the per-lane blocks of runs (R even, R = 2 mod 4 from 8 on, at most 32 blocks),
  - values accumulated relative to the run before each block, with the block's offset taken from
    a scan of the blocks' sums of l afterwards,
  - pairs past a block's end evaluated with l = 0 and the block's last C (no effect),
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


def lane_blocks(Uc):
    Ue = Uc + (Uc & 1)
    R = (Ue + 31) // 32
    R += R & 1
    if R >= 8 and R % 4 == 0:
        R += 2
    return Ue, R, [(min(L * R, Ue), min(min(L * R, Ue) + R, Ue)) for L in range(32)]


def sweep_g(x, m, lo, hi, A, B):
    """The sweep's arithmetic: compact runs, lane blocks, relative values, block-sum scan."""
    dv = np.unique(x)
    rk = np.searchsorted(dv, x)
    H = hi - lo
    cnt = np.bincount(rk[lo * m:hi * m], minlength=len(dv))
    keep = np.nonzero(cnt)[0]
    mp = np.full(len(dv), -1)
    mp[keep] = np.arange(len(keep))
    Uc = len(keep)
    Ue, R, blocks = lane_blocks(Uc)
    assert R <= 50 and all(b1 - b0 <= R and (b1 - b0) % 2 == 0 for b0, b1 in blocks)
    C = [int(c) % M32 for c in np.cumsum(cnt[keep])]
    if Uc & 1:
        C.append(C[-1])  # padding run: l = 0, same C
    l = [0] * Ue

    def add_step(t):
        for j in range(m):
            c = mp[rk[t * m + j]]
            l[c] = (l[c] + H) % M32

    for t in range(lo, A):
        add_step(t)
    res = {}
    for k in range(A, B + 1):
        a = k - lo
        sums, ext = [], []
        for b0, b1 in blocks:
            Cb = C[b0 - 1] if b0 > 0 else 0
            clast = C[b1 - 1] if b1 > b0 else 0
            h0 = (a * Cb) % M32
            hc, mx, mn = h0, -(1 << 31), (1 << 31) - 1
            npair = (b1 - b0) // 2
            for g in range(0, 25, 4):  # groups of four pairs, as loaded
                if g >= npair:
                    break
                for j in range(g, min(g + 4, 25)):
                    lo2 = (l[b0 + 2 * j], l[b0 + 2 * j + 1]) if j < npair else (0, 0)
                    c0 = C[b0 + 2 * j] if b0 + 2 * j < b1 else clast
                    c1 = C[b0 + 2 * j + 1] if b0 + 2 * j + 1 < b1 else clast
                    hc = (hc + lo2[0]) % M32
                    v0 = s32(hc + (M32 - a) * c0)
                    hc = (hc + lo2[1]) % M32
                    v1 = s32(hc + (M32 - a) * c1)
                    mx, mn = max(mx, v0, v1), min(mn, v0, v1)
            sums.append((hc - h0) % M32)
            ext.append((Cb, mx, mn, npair > 0))
        carry, g = 0, 0
        for blk, (Cb, mx, mn, nonempty) in zip(sums, ext):
            vs = (carry - a * Cb) % M32
            if nonempty:
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
    """Blocks tile [0, Ue) in at most 32 lanes, R <= 50, and, from R = 8 on, a half warp's 8-byte
    pair loads fall on distinct banks (R = 2 mod 4)."""
    for Uc in range(1, 1537):
        Ue, R, blocks = lane_blocks(Uc)
        covered = [c for b0, b1 in blocks for c in range(b0, b1)]
        assert covered == list(range(Ue))
        assert R <= 50
        if R >= 8:
            banks = {((L * R) // 2) % 16 for L in range(16)}
            assert len(banks) == 16


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
