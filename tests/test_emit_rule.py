"""The key emission's split of output slots over warps (bin.cu, k_emit_keys),
restated in numpy: warp w takes slots [512 w, 512 (w + 1)), finds the pair
holding its first slot by a 32-way search of the offsets, keeps a window of
32 consecutive pairs, moves it when a round of 32 slots runs past it, and
looks a slot up in the offsets directly when the window cannot hold it
(pairs without fragments).  Every slot must land on the pair and the local
index that a plain expansion of the counts gives, for counts with huge
pairs, runs of single fragments and runs of empty pairs."""
import numpy as np

SLOTS = 512


def first_pair(offsets, n, fb):
    lo, hi = 0, n
    while hi - lo > 32:
        step = (hi - lo + 31) // 32
        q = lo + np.arange(32) * step
        ok = (q < hi) & (offsets[np.minimum(q, n - 1)] <= fb)
        L = int(np.nonzero(ok)[0].max())
        lo = lo + L * step
        hi = min(lo + step, hi)
    q = lo + np.arange(32)
    ok = (q < hi) & (offsets[np.minimum(q, n - 1)] <= fb)
    return lo + int(np.nonzero(ok)[0].max())


def window(offsets, counts, n, F, pw):
    p = pw + np.arange(32)
    valid = p < n
    start = np.where(valid, offsets[np.minimum(p, n - 1)], F)
    cnt = np.where(valid, counts[np.minimum(p, n - 1)], 0)
    return start, cnt


def emit(counts):
    n = len(counts)
    offsets = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
    F = int(counts.sum())
    pair = np.full(F, -1, np.int64)
    local = np.full(F, -1, np.int64)
    for w in range((F + SLOTS - 1) // SLOTS):
        fb = w * SLOTS
        f_end = min(fb + SLOTS, F)
        pw = first_pair(offsets, n, fb)
        start, cnt = window(offsets, counts, n, F, pw)
        for fr in range(fb, f_end, 32):
            last = min(fr + 31, f_end - 1)
            if last >= start[31] + cnt[31]:
                pw += int(np.nonzero(start <= fr)[0].max())
                start, cnt = window(offsets, counts, n, F, pw)
            for lane in range(32):
                f = fr + lane
                if f >= f_end:
                    continue
                L = int(np.nonzero(start <= f)[0].max())
                p, s, c = pw + L, start[L], cnt[L]
                if f - s >= c:                    # past the window: the offsets directly
                    p = int(np.searchsorted(offsets, f, side="right") - 1)
                    s, c = offsets[p], counts[p]
                assert f - s < c
                pair[f], local[f] = p, f - s
    return pair, local


def plain(counts):
    pair = np.repeat(np.arange(len(counts)), counts)
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    return pair, np.arange(len(pair)) - starts[pair]


def test_slot_split_matches_the_plain_expansion():
    rng = np.random.default_rng(0)
    cases = [
        rng.integers(1, 6, 3000),                                       # small pairs
        np.concatenate([np.full(64, 1200), rng.integers(1, 6, 2000)]),  # huge pairs first
        np.concatenate([rng.integers(1, 4, 500), np.zeros(200, np.int64), rng.integers(1, 40, 500)]),  # empty run
        np.array([5000]),                                               # one pair
        np.concatenate([np.zeros(40, np.int64), [7], np.zeros(70, np.int64), [3, 1]]),
    ]
    for counts in cases:
        counts = counts.astype(np.int64)
        pair, local = emit(counts)
        p0, l0 = plain(counts)
        assert np.array_equal(pair, p0) and np.array_equal(local, l0)
