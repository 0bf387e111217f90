"""The index arithmetic of the sampler's search primitives (csrc/device.cuh),
transcribed step for step and run on the CPU: every read stays inside the
searched list and the answer is right, for every list length up to 300 and
every key below, between and above the elements.  A per-lane halving search
keeps b + n <= len (its first read b + n/2 < b + n, its last b < len); the
warp's 32-ary upper bound reads a slot only below its open upper end, which
never grows.  CPU only."""
import numpy as np
import pytest


def lane_contains(a, x, reads):
    n = len(a)
    if n == 0:
        return False
    b = 0
    while n > 1:
        half = n >> 1
        reads.append(b + half)
        b = b + half if a[b + half] <= x else b
        n -= half
    reads.append(b)
    return a[b] == x


def lane_find(a, x, reads):
    n = len(a)
    if n == 0:
        return None
    b = 0
    while n > 1:
        half = n >> 1
        reads.append(b + half)
        b = b + half if a[b + half] <= x else b
        n -= half
    reads.append(b)
    return b if a[b] == x else None


def warp_upper_bound(a, key, reads):
    lo, hi = 0, len(a)
    while hi - lo > 32:
        step = (hi - lo + 31) // 32
        le = []
        for lane in range(32):
            pos = lo + lane * step
            ok = pos < hi
            if ok:
                reads.append(pos)
                ok = a[pos] <= key
            le.append(ok)
        c = sum(le)
        assert le == [True] * c + [False] * (32 - c)     # the true lanes form a prefix
        if c == 0:
            return lo
        nlo = lo + (c - 1) * step + 1
        nhi = lo + c * step
        lo, hi = nlo, min(nhi, hi)
    c = 0
    for lane in range(32):
        pos = lo + lane
        if pos < hi:
            reads.append(pos)
            c += a[pos] <= key
    return lo + c


@pytest.mark.parametrize("seed", [0, 1])
def test_searches_stay_inside_the_list(seed):
    rng = np.random.default_rng(seed)
    for n in list(range(0, 70)) + list(range(70, 300, 7)) + [1023, 1024, 1025, 4097]:
        a = np.sort(rng.choice(10 * n + 10, size=n, replace=False)).tolist()
        keys = sorted(set([-1, 10 * n + 11] + a + [v + 1 for v in a] + [v - 1 for v in a]))
        if n > 300:
            keys = keys[::max(1, len(keys) // 200)]
        for x in keys:
            reads = []
            assert lane_contains(a, x, reads) == (x in a)
            assert all(0 <= r < n for r in reads)
            reads = []
            f = lane_find(a, x, reads)
            assert f == (a.index(x) if x in a else None)
            assert all(0 <= r < n for r in reads)
            reads = []
            assert warp_upper_bound(a, x, reads) == int(np.searchsorted(a, x, side="right"))
            assert all(0 <= r < n for r in reads)
