"""The index arithmetic of the sampler's search primitives (csrc/device.cuh)
and of its windowed partner staging (csrc/sampler.cuh), transcribed step for
step and run on the CPU: every read stays inside the searched list and the
answer is right, for every list length up to 300 and every key below, between
and above the elements.  A per-lane halving search keeps b + n <= len (its
first read b + n/2 < b + n, its last b < len); the warp's 32-ary upper bound
reads a slot only below its open upper end, which never grows (the 32-bit form
computes the piece length as ((hi - lo - 1) >> 5) + 1, the same ceiling).
The windowed staging settles every driver entry exactly once, in order, and
reads the partner only inside its list; the vertex-induced single-list step
counts |S_j| and draws S_j's t-th entry from the positions of the removed
entries alone.  CPU only."""
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


def warp_upper_bound(a, key, reads, form32=False):
    lo, hi = 0, len(a)
    while hi - lo > 32:
        step = (((hi - lo - 1) >> 5) + 1) if form32 else (hi - lo + 31) // 32
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
            for form32 in (False, True):
                reads = []
                assert warp_upper_bound(a, x, reads, form32) == int(np.searchsorted(a, x, side="right"))
                assert all(0 <= r < n for r in reads)


def windowed_intersection(D, Q, cap, reads_q, reads_d):
    """The compact sampler's step-2 loop with the partner Q (longer than the
    buffer) staged in windows of cap entries: each window settles the driver
    entries up to its last element (all of them in the last window), in
    groups of 32 lanes read 128 at a time."""
    dlen, qn = len(D), len(Q)
    out = []
    pw, dcur = 0, 0
    while True:
        wn = min(qn - pw, cap)
        assert wn >= 1
        win = []
        for idx in range(wn):
            reads_q.append(pw + idx)
            win.append(Q[pw + idx])
        pw += wn
        tail = pw >= qn
        wlast = win[-1]
        stop = False
        base = dcur
        while base < dlen and not stop:
            for u in range(4):
                b = base + 32 * u
                if b >= dlen:
                    break
                ins = []
                for lane in range(32):
                    idx = b + lane
                    y = None
                    if idx < dlen:
                        reads_d.append(idx)
                        y = D[idx]
                    inside = idx < dlen and (tail or y <= wlast)
                    ins.append(inside)
                    if inside and y in win:
                        out.append(y)
                if not tail:
                    c = sum(ins)
                    assert ins == [True] * c + [False] * (32 - c)   # a prefix
                    if c < 32:
                        dcur = b + c
                        stop = True
                        break
            base += 128
        if tail or not stop:
            break
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_windowed_partner_staging_settles_every_driver_entry_once(seed):
    rng = np.random.default_rng(seed)
    for trial in range(60):
        universe = int(rng.integers(50, 5000))
        dlen = int(rng.integers(1, min(universe, 400)))
        qn = int(rng.integers(1, min(universe, 1500)))
        D = np.sort(rng.choice(universe, size=dlen, replace=False)).tolist()
        Q = np.sort(rng.choice(universe, size=qn, replace=False)).tolist()
        for cap in (1, 7, 32, 64, 100, 832):
            if qn <= cap:
                continue
            rq, rd = [], []
            got = windowed_intersection(D, Q, cap, rq, rd)
            assert got == sorted(set(D) & set(Q))
            assert all(0 <= r < qn for r in rq) and all(0 <= r < dlen for r in rd)
            assert len(set(rq)) == len(rq)     # every partner entry staged at most once


def induced_positions_draw(A, nn_lists, matched, t):
    """The vertex-induced single-list step, transcribed: the positions in A of
    the entries of each non-neighbour list (one ascending run per list, an
    entry counted in the first list holding it, matched vertices left out),
    the positions of the matched vertices in A apart, |S| = |A| - removed, and
    the drawn position by the fixed point idx = t + #(removed <= idx)."""
    pos = {y: q for q, y in enumerate(A)}
    amax = A[-1]
    runs = []
    for i, B in enumerate(nn_lists):
        run = []
        for y in B:
            if y > amax:
                break
            q = pos.get(y)
            if q is None or y in matched:
                continue
            if any(y in set(nn_lists[i2]) for i2 in range(i)):
                continue
            run.append(q)
        assert run == sorted(run) and len(set(run)) == len(run)
        runs.append(run)
    qm = [pos[v] for v in matched if v in pos]
    removed = sum(len(r) for r in runs) + len(qm)
    count = len(A) - removed
    if count == 0:
        return count, None
    assert 0 <= t < count
    idx = t
    while True:
        c = sum(int(np.searchsorted(r, idx, side="right")) for r in runs) + sum(q <= idx for q in qm)
        nx = t + c
        if nx == idx:
            break
        idx = nx
    assert 0 <= idx < len(A)
    return count, idx


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_induced_single_list_positions_draw_the_right_entry(seed):
    rng = np.random.default_rng(seed)
    for trial in range(200):
        universe = int(rng.integers(20, 400))
        A = sorted(rng.choice(universe, size=int(rng.integers(1, universe // 2 + 1)), replace=False).tolist())
        nn_lists = [sorted(rng.choice(universe + 50, size=int(rng.integers(0, 40)), replace=False).tolist())
                    for _ in range(int(rng.integers(1, 4)))]
        matched = set(rng.choice(universe, size=int(rng.integers(0, 4)), replace=False).tolist())
        removed = set().union(*[set(b) for b in nn_lists]) | matched
        S = [y for y in A if y not in removed]
        for t in range(len(S)):
            count, idx = induced_positions_draw(A, nn_lists, matched, t)
            assert count == len(S) and A[idx] == S[t]
        if not S:
            assert induced_positions_draw(A, nn_lists, matched, 0) == (0, None)
