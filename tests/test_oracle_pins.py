"""Pins of the CPU oracle against facts fixed outside it: published known-answer
vectors, a library routine, closed forms, brute force on tiny graphs, exact
enumeration of the sampling tree, and statistics over many seeds.

These run on CPU only (no GPU, no CUDA library)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

from oracle import brute
from oracle import oracle as O
from paper_2405_03488_gb300 import graphs as G

HERE = os.path.dirname(os.path.abspath(__file__))


def og(rp, col):
    return O.Graph(*G.to_numpy(rp, col))


# ------------------------------------------------------------------ Philox
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert O.philox(v[0:4], v[4:6]) == tuple(v[6:10])


def test_choice_word_counter_layout():
    # choice t of sample s: word pair (t mod 2) of the block with counter
    # (s_lo, s_hi, t // 2, slot << 8 | purpose) under key (seed_lo, seed_hi)
    seed, s = 0x1234_5678_9ABC_DEF0, (7 << 32) | 99
    for t in range(6):
        for slot, purpose in ((0, 0), (3, 0), (0, 2)):
            o = O.philox((s & 0xFFFFFFFF, s >> 32, t // 2, (slot << 8) | purpose),
                         (seed & 0xFFFFFFFF, seed >> 32))
            w = 2 * (t % 2)
            assert O.choice_word(seed, s, t, slot, purpose) == o[w] | (o[w + 1] << 32)


def test_index_map_is_multiply_high():
    rng = np.random.default_rng(0)
    for _ in range(2000):
        r = int(rng.integers(0, 2**64, dtype=np.uint64))
        n = int(rng.integers(1, 2**63, dtype=np.uint64)) >> int(rng.integers(0, 62))
        n = max(n, 1)
        assert O.index_map(r, n) == (r * n) >> 64
    assert O.index_map(2**64 - 1, 10) == 9
    assert O.index_map(0, 10) == 0


# ------------------------------------------------------------------ Phi^-1
def test_phi_inv_matches_scipy():
    from scipy.special import ndtri
    ps = np.concatenate([np.logspace(-300, -1, 200), np.linspace(0.01, 0.99, 199),
                         1 - np.logspace(-15, -2, 50)])
    for p in ps:
        a, b = O.phi_inv(float(p)), float(ndtri(p))
        assert abs(a - b) <= 2e-15 * max(1.0, abs(b)), (p, a, b)
    assert O.phi_inv(1 - 0.01 / 2) == pytest.approx(2.5758293035489004, rel=1e-15)
    assert O.phi_inv(1 - 0.05 / 2) == pytest.approx(1.959963984540054, rel=1e-15)


# ------------------------------------------------------------------ plan
ALL_PATTERNS = ["triangle", "wedge", "3-star", "4-path", "tailed-triangle", "4-cycle", "diamond",
                "4-clique", "5-clique", "5-path", "house", "dumbbell", "6-clique"]


@pytest.mark.parametrize("name", ALL_PATTERNS + ["7-clique", "8-clique", "9-clique"])
def test_plan_aut_size_matches_brute_force(name):
    k, edges = G.pattern(name)
    p = O.plan(k, edges)
    if k <= 7:
        assert p.aut_size == brute.automorphisms(k, edges)
    else:
        assert p.aut_size == math.factorial(k)   # cliques: the full symmetric group
    # matching order: every later vertex has a back-neighbour
    for j in range(1, k):
        assert p.adj[j] & ((1 << j) - 1)


@pytest.mark.parametrize("k", [3, 4, 5, 6, 7, 8, 9])
def test_plan_clique_is_total_order(k):
    p = O.plan(*G.clique(k))
    assert set(p.restrictions()) == {(i, j) for i in range(k) for j in range(i + 1, k)}
    assert p.oriented == 1


def test_plan_four_cycle_matches_algorithm4_mirror():
    # Algorithm 4 breaks the 4-cycle's symmetry with v0 the extreme vertex and
    # v3 < v1; with '<' pinned the order 0-1-2-3 gets v0 < v1, v2, v3 and v1 < v3
    p = O.plan(*G.pattern("4-cycle"))
    assert set(p.restrictions()) == {(0, 1), (0, 2), (0, 3), (1, 3)}
    assert p.oriented == 1


def test_plan_rejects_disconnected():
    with pytest.raises(ValueError):
        O.plan(4, [(0, 1), (2, 3)])


# ------------------------------------------------------------------ exact counts
def small_graphs():
    out = [("K6", G.complete(6)), ("K33", G.complete_bipartite(3, 3)), ("star5", G.star(5)),
           ("C7", G.cycle(7))]
    for seed in range(4):
        out.append(("er%d" % seed, G.random_small(9, 0.5, seed + 10)))
    return out


@pytest.mark.parametrize("name", ALL_PATTERNS[:11])
@pytest.mark.parametrize("induced", [False, True])
def test_exact_count_matches_brute_force(name, induced):
    k, edges = G.pattern(name)
    p = O.plan(k, edges, induced)
    for gname, (rp, col) in small_graphs():
        g = og(rp, col)
        want = brute.count(*G.to_numpy(rp, col), k, edges, induced)
        assert O.exact_count(g, p) == want, (gname, name, induced)


def test_closed_forms():
    for n in (5, 7, 9):
        g = og(*G.complete(n))
        for k in (3, 4, 5):
            assert O.exact_count(g, O.plan(*G.clique(k))) == math.comb(n, k)
    for a, b in ((2, 3), (3, 4), (4, 5)):
        g = og(*G.complete_bipartite(a, b))
        assert O.exact_count(g, O.plan(*G.pattern("4-cycle"))) == math.comb(a, 2) * math.comb(b, 2)
        assert O.exact_count(g, O.plan(*G.pattern("triangle"))) == 0
    for leaves in (3, 6, 9):
        g = og(*G.star(leaves))
        assert O.exact_count(g, O.plan(*G.pattern("3-star"))) == math.comb(leaves, 3)
        assert O.exact_count(g, O.plan(*G.pattern("triangle"))) == 0
    for n in (5, 8, 11):
        g = og(*G.cycle(n))
        assert O.exact_count(g, O.plan(*G.pattern("4-cycle"))) == 0
        assert O.exact_count(g, O.plan(*G.pattern("4-path"))) == n
    rp, col = G.random_small(12, 0.4, 3)
    deg = np.diff(rp.numpy())
    assert O.exact_count(og(rp, col), O.plan(*G.pattern("wedge"))) == sum(math.comb(int(d), 2) for d in deg)


# ------------------------------------------------------------------ sampling tree
def _ceil_word(i, n):
    return -((-(i << 64)) // n)


def enumerate_tree(g, p, mode, mlp=None):
    """Every path of the sampler, driven by explicit choice words: returns the
    hit leaves as (vertices, probability, record) and the total probability."""
    k = p.k
    M = g.m if (p.oriented and mode != O.LAZY) else g.nnz
    leaves = []
    total = [Fraction(0)]

    def walk(r, j, prob):
        if j == k:
            return
        rr = r + [0] * (k - 1 - len(r))
        rec = O.sample(g, p, rr, mode, mlp)
        if mode == O.LEARNED and j <= k - 2 and rec.aux[j] > 0:
            A = rec.factor[j]
            t = 0
            while t < A:
                w = _ceil_word(t, A)
                rec = O.sample(g, p, r + [w] + [0] * (k - 2 - len(r)), mode, mlp)
                a = rec.aux[j]
                branch(r + [w], j, prob * Fraction(a, A), rec)
                t += a
            return
        size = rec.factor[j]
        if size == 0:
            total[0] += prob
            return
        for i in range(size):
            w = _ceil_word(i, size)
            rec = O.sample(g, p, r + [w] + [0] * (k - 2 - len(r)), mode, mlp)
            branch(r + [w], j, prob / size, rec)

    def branch(r, j, prob, rec):
        if rec.hit and j == k - 1:
            leaves.append((tuple(rec.vert[:k]), prob, rec))
            total[0] += prob
        elif (rec.hit or rec.depth > j) and j < k - 1:
            walk(r, j + 1, prob)
        else:
            total[0] += prob

    for e in range(M):
        w0 = _ceil_word(e, M)
        rec = O.sample(g, p, [w0] + [0] * (k - 2), mode, mlp)
        if k == 2:
            leaves.append((tuple(rec.vert[:2]), Fraction(1, M), rec))
            total[0] += Fraction(1, M)
        else:
            walk([w0], 2, Fraction(1, M))
    return leaves, total[0]


def leaf_weight(rec, k, mode):
    w = Fraction(int(rec.factor[0]))
    for j in range(2, k):
        if mode == O.LEARNED and j <= k - 2 and rec.aux[j] > 0:
            w *= Fraction(int(rec.factor[j]), int(rec.aux[j]))
        else:
            w *= int(rec.factor[j])
    return w


def as_match(verts, k, edges, order):
    # vertex of pattern position j is verts[j]; map pattern edges through the order
    pos = {order[j]: j for j in range(k)}
    vs = frozenset(verts)
    es = frozenset(frozenset((verts[pos[a]], verts[pos[b]])) for a, b in edges)
    return vs, es


def random_mlp(seed):
    rng = np.random.default_rng(seed)

    def bf16(a):
        a = np.asarray(a, dtype=np.float32)
        return (a.view(np.uint32) >> 16).astype(np.uint16)

    return O.Weights16(bf16(rng.normal(0, 0.8, (64, 3))), bf16(rng.normal(0, 0.3, 64)),
                       bf16(rng.normal(0, 0.2, (64, 64))), bf16(rng.normal(0, 0.1, 64)),
                       bf16(rng.normal(0, 0.3, 64)), bf16([0.1]))


TREE_CASES = [("triangle", False), ("4-clique", False), ("4-cycle", False), ("4-cycle", True),
              ("diamond", False), ("tailed-triangle", True), ("3-star", False), ("4-path", True),
              ("house", False), ("5-clique", False),
              # edge-induced patterns with single-back-neighbour steps
              ("wedge", False), ("4-path", False), ("5-path", False), ("dumbbell", False)]


@pytest.mark.parametrize("name,induced", TREE_CASES)
@pytest.mark.parametrize("mode", [O.INTERSECT, O.CHECK, O.LEARNED, O.LAZY])
def test_sampling_tree_is_exact(name, induced, mode):
    """Lemma 1: each match is reached by exactly one path, whose probability is
    the inverse of its weight; so the hit leaves are exactly the matches and
    E[X] = sum over hit leaves of Pr * w = C with no statistics involved."""
    k, edges = G.pattern(name)
    p = O.plan(k, edges, induced)
    mlp = random_mlp(7) if mode == O.LEARNED else None
    for gname, (rp, col) in small_graphs()[:6]:
        g = og(rp, col)
        leaves, total = enumerate_tree(g, p, mode, mlp)
        assert total == 1, (gname, total)
        want = brute.matches(*G.to_numpy(rp, col), k, edges, induced)
        got = [as_match(v, k, edges, list(p.order)) for v, _, _ in leaves]
        assert len(got) == len(set(got)), "a match reached by two paths"
        assert set(got) == want, gname
        for _, prob, rec in leaves:
            w = leaf_weight(rec, k, mode)
            assert prob * w == 1
            assert rec.w_f64 == pytest.approx(float(w), rel=1e-15)
            if mode != O.LEARNED:
                assert rec.w_u64 == w and rec.w_f64 == float(w)


def exact_moments(g, p, mode, mlp=None):
    leaves, _ = enumerate_tree(g, p, mode, mlp)
    mean = sum(prob * leaf_weight(rec, p.k, mode) for _, prob, rec in leaves)
    ex2 = sum(prob * leaf_weight(rec, p.k, mode) ** 2 for _, prob, rec in leaves)
    return mean, ex2 - mean * mean


@pytest.mark.parametrize("name,induced,mode", [("4-clique", False, O.INTERSECT),
                                               ("4-cycle", False, O.CHECK),
                                               ("4-cycle", False, O.LAZY),
                                               ("tailed-triangle", True, O.LAZY),
                                               ("house", False, O.INTERSECT),
                                               ("diamond", True, O.LEARNED)])
def test_unbiased_over_philox_samples(name, induced, mode):
    k, edges = G.pattern(name)
    p = O.plan(k, edges, induced)
    mlp = random_mlp(3) if mode == O.LEARNED else None
    rp, col = G.random_small(10, 0.55, 21)
    g = og(rp, col)
    mean, var = exact_moments(g, p, mode, mlp)
    C = brute.count(*G.to_numpy(rp, col), k, edges, induced)
    assert mean == C
    N = 200_000
    acc, _ = O.ns_run(g, p, seed=5, first=0, count=N, mode=mode, mlp=mlp)
    est = acc.sum / N
    z = (est - C) / math.sqrt(float(var) / N)
    assert abs(z) < 5.0, (est, C, z)
    # the sample variance approaches the exact per-sample variance
    sv = acc.sumsq / N - est * est
    assert sv == pytest.approx(float(var), rel=0.1)


def test_sums_match_exact_integer_sums():
    rp, col = G.random_small(12, 0.5, 5)
    g = og(rp, col)
    p = O.plan(*G.clique(4))
    acc, recs = O.ns_run(g, p, seed=9, first=1000, count=50_000, trace=True)
    w = [int(x) for x in recs["w_u64"]]
    assert all(int(r["w_f64"]) == int(r["w_u64"]) for r in recs)
    assert acc.n == 50_000 and acc.hits == int(recs["hit"].sum())
    assert acc.sum == pytest.approx(sum(w), rel=1e-12)
    assert acc.sumsq == pytest.approx(sum(x * x for x in w), rel=1e-12)


def test_er_expected_triangles():
    # G(n, p): E[triangles] = C(n,3) p^3; with n=400, p=0.05 the count has a
    # standard deviation of about 10% of the mean
    n, pr = 400, 0.05
    counts = []
    for seed in range(8):
        g = og(*G.erdos_renyi(n, pr, seed=seed + 100))
        counts.append(O.exact_count(g, O.plan(*G.pattern("triangle"))))
    want = math.comb(n, 3) * pr ** 3
    assert np.mean(counts) == pytest.approx(want, rel=0.12)


# ------------------------------------------------------------------ online convergence
def test_error_of_closed_form():
    z = O.phi_inv(0.995)
    # samples {0, 0, 0, 4}: mean 1, population variance 3, sigma = sqrt(3/4)
    mu, half, eh = O.error_of(4.0, 16.0, 4, z)
    assert mu == 1.0
    assert half == pytest.approx(z * math.sqrt(3 / 4), rel=1e-15)
    assert eh == pytest.approx(z * math.sqrt(3 / 4), rel=1e-15)
    mu, half, eh = O.error_of(0.0, 0.0, 10, z)
    assert mu == 0.0 and eh == math.inf
    mu, half, eh = O.error_of(50.0, 250.0, 10, z)      # all samples equal 5
    assert mu == 5.0 and half == 0.0 and eh == 0.0


def test_online_stops_at_once_on_constant_weights():
    # the one-edge pattern has weight m on every sample: zero variance, so the
    # first window already gives eps_hat = 0 and the exact count
    g = og(*G.complete(7))
    p = O.plan(*G.pattern("edge"))
    out = O.ns_online(g, p, eps=0.01, delta=0.01, seed=1, window=64)
    assert out.converged == 1 and out.rounds == 1 and out.samples == 64
    assert out.estimate == 21.0 and out.eps_hat == 0.0


def test_online_window_and_stop_rule():
    rp, col = G.random_small(12, 0.5, 8)
    g = og(rp, col)
    p = O.plan(*G.clique(4))
    W = 4096
    out = O.ns_online(g, p, eps=0.05, delta=0.05, seed=3, window=W)
    assert out.converged == 1
    assert out.samples == out.rounds * W
    # the same prefix of samples reproduces the statistics
    acc, _ = O.ns_run(g, p, seed=3, first=0, count=out.samples)
    z = O.phi_inv(1 - 0.05 / 2)
    mu, half, eh = O.error_of(acc.sum, acc.sumsq, acc.n, z)
    assert (mu, half, eh) == (out.estimate, out.ci_half_width, out.eps_hat)
    assert eh <= 0.05
    if out.rounds > 1:
        acc2, _ = O.ns_run(g, p, seed=3, first=0, count=out.samples - W)
        assert O.error_of(acc2.sum, acc2.sumsq, acc2.n, z)[2] > 0.05
    # n_max stops an unconverged run
    out2 = O.ns_online(g, p, eps=1e-6, delta=0.05, seed=3, window=W, n_max=3 * W)
    assert out2.converged == 0 and out2.samples == 3 * W


def test_online_interval_coverage_over_seeds():
    """Empirical coverage of the convergence test (Algorithm 3, Theorem 1): over
    400 seeds the stopped estimate misses C by more than eps C in at most
    delta R runs plus three binomial standard deviations."""
    rp, col = G.erdos_renyi(300, 0.08, seed=21)
    g = og(rp, col)
    R, eps, delta, W = 400, 0.1, 0.05, 1 << 9
    for name in ("triangle", "4-cycle"):
        p = O.plan(*G.pattern(name))
        C = O.exact_count(g, p)
        miss = 0
        for s in range(1, R + 1):
            o = O.ns_online(g, p, eps, delta, seed=s, window=W)
            assert o.converged == 1
            miss += abs(o.estimate - C) > eps * C
        assert miss <= R * delta + 3 * (R * delta * (1 - delta)) ** 0.5, (name, miss)


# ------------------------------------------------------------------ GS
def test_gs_one_colour_is_exact():
    rp, col = G.random_small(11, 0.5, 2)
    g = og(rp, col)
    for name in ("triangle", "4-clique", "4-cycle", "house"):
        p = O.plan(*G.pattern(name))
        est, cp = O.gs_estimate(g, p, c=1, seed=4)
        assert cp == O.exact_count(g, p) and est == float(cp)


def test_gs_expectation_over_all_colourings_is_exact():
    """Colour sparsification keeps a k-vertex match iff all k vertices share a
    colour (probability c^-(k-1)), so averaging C' c^(k-1) over every colouring
    gives C exactly."""
    import itertools
    rp, col = G.random_small(8, 0.6, 6)
    g = og(rp, col)
    for name, c in (("triangle", 2), ("4-clique", 2), ("4-cycle", 2), ("triangle", 3)):
        p = O.plan(*G.pattern(name))
        C = O.exact_count(g, p)
        tot = 0
        n_col = 0
        for cols in itertools.product(range(c), repeat=g.n):
            row, cc = O.sparsify(g, np.array(cols, dtype=np.uint32))
            tot += O.exact_count(O.Graph(row, cc), p)
            n_col += 1
        assert Fraction(tot * c ** (p.k - 1), n_col) == C, name


def test_colour_is_word0_of_purpose2_block():
    seed, c = 77, 8
    cols = O.colors(50, c, seed, colouring=3)
    for v in range(50):
        w0 = O.philox((v, 0, 3, 2), (seed, 0))[0]
        assert cols[v] == (w0 * c) >> 32
    big = O.colors(40000, c, seed)
    frac = np.bincount(big, minlength=c) / len(big)
    assert np.all(np.abs(frac - 1 / c) < 0.01)


def test_sparsify_keeps_monochromatic_edges():
    rp, col = G.random_small(12, 0.5, 9)
    g = og(rp, col)
    cols = O.colors(g.n, 3, 5)
    row, cc = O.sparsify(g, cols)
    want = [(u, int(x)) for u in range(g.n) for x in col[rp[u]:rp[u + 1]].numpy() if cols[u] == cols[x]]
    got = [(u, int(x)) for u in range(g.n) for x in cc[row[u]:row[u + 1]]]
    assert got == want
    assert O.validate(row, cc) == 0


def test_bes_expectation_over_all_edge_subsets_is_exact():
    """Bernoulli edge sparsification with p = 1/2: every subset of the m edges is
    equally likely, and a match survives iff its l edges all stay, so the mean
    of C' over all 2^m subsets is C 2^-l exactly (Algorithm 2: scale by p^-l,
    l the pattern's edge count, not k - 1)."""
    import itertools
    rp, col = G.random_small(7, 0.55, 4)
    rp, col = G.to_numpy(rp, col)
    edges = [(u, int(x)) for u in range(len(rp) - 1) for x in col[rp[u]:rp[u + 1]] if u < x]
    m = len(edges)
    assert 8 <= m <= 14
    g = O.Graph(rp, col)
    for name in ("triangle", "4-cycle", "4-path", "diamond"):
        k, pe = G.pattern(name)
        p = O.plan(k, pe)
        C = O.exact_count(g, p)
        tot = 0
        for keep in itertools.product((0, 1), repeat=m):
            adj = [[] for _ in range(len(rp) - 1)]
            for (u, w), kk in zip(edges, keep):
                if kk:
                    adj[u].append(w)
                    adj[w].append(u)
            row = np.zeros(len(rp), dtype=np.uint64)
            cc = []
            for u, a in enumerate(adj):
                cc += sorted(a)
                row[u + 1] = len(cc)
            tot += O.exact_count(O.Graph(row, np.array(cc, dtype=np.uint32)), p)
        assert Fraction(tot, 2 ** m) == Fraction(C, 2 ** len(pe)), name


def test_bes_keep_is_word0_of_purpose3_block_on_the_unordered_pair():
    seed = 123
    assert O.bes_threshold(0.3) == 1288490188 and O.bes_threshold(1.0) == 1 << 32
    assert O.bes_threshold(0.5) == 1 << 31
    t = O.bes_threshold(0.3)
    for (u, w) in ((0, 1), (7, 3), (100, 5), (2 ** 32 - 2, 17)):
        lo, hi = min(u, w), max(u, w)
        w0 = O.philox((lo, hi, 2, (5 << 8) | 3), (seed, 0))[0]
        assert O.bes_keep(seed, u, w, t, colouring=2, slot=5) == (w0 < t)
        assert O.bes_keep(seed, u, w, t, colouring=2, slot=5) == O.bes_keep(seed, w, u, t, colouring=2, slot=5)
    rng = np.random.default_rng(1)
    pairs = rng.integers(0, 1 << 20, size=(60000, 2))
    frac = np.mean([O.bes_keep(seed, int(a), int(b), t) for a, b in pairs])
    assert abs(frac - t / 2 ** 32) < 0.008            # 4 binomial standard deviations
    assert all(O.bes_keep(seed, int(a), int(b), 1 << 32) for a, b in pairs[:200])


def test_bes_sparsify_keeps_each_edge_once_for_both_directions():
    rp, col = G.random_small(30, 0.4, 5)
    g = og(rp, col)
    t = O.bes_threshold(0.45)
    row, cc = O.bes_sparsify(g, 9, t, colouring=1, slot=2)
    assert O.validate(row, cc) == 0                    # symmetric, sorted, no loops
    want = [(u, int(x)) for u in range(g.n) for x in col[rp[u]:rp[u + 1]].numpy()
            if O.bes_keep(9, u, int(x), t, colouring=1, slot=2)]
    got = [(u, int(x)) for u in range(g.n) for x in cc[row[u]:row[u + 1]]]
    assert got == want


# ------------------------------------------------------------------ validation
def test_validate_detects_each_violation():
    rp, col = G.to_numpy(*G.complete(4))
    assert O.validate(rp, col) == 0
    bad = col.copy(); bad[0] = 9
    assert O.validate(rp, bad) == -2
    bad = col.copy(); bad[0] = 0
    assert O.validate(rp, bad) == -3
    bad = col.copy(); bad[0], bad[1] = bad[1], bad[0]
    assert O.validate(rp, bad) == -4
    # asymmetric: drop one direction
    rp2 = np.array([0, 1, 1], dtype=np.uint64)
    assert O.validate(rp2, np.array([1], dtype=np.uint32)) == -5


# ------------------------------------------------------------------ learned proposal
def test_flog2p1_pins():
    for e in range(0, 40):
        assert O.flog2p1(2**e - 1) == float(e)          # exact at powers of two
    prev = -1.0
    for d in range(0, 5000):
        f = O.flog2p1(d)
        assert f > prev
        assert abs(f - math.log2(1 + d)) <= 0.0861   # max gap of the chord below log2
        prev = f


def test_score_mapping():
    assert O.score(-100.0) == 1
    assert O.score(float("nan")) == 1
    assert O.score(100.0) == 4097
    assert O.score(0.0) == 1 + 2048
    assert O.score(4.0) == 4097
    assert O.score(-4.0) == 1


def test_mlp_logit_matches_torch_float64():
    mlp = random_mlp(11)
    ws = [torch.from_numpy((a.astype(np.uint32) << 16).view(np.float32)).double() for a in mlp.arrs]
    w1, b1, w2, b2, w3, b3 = ws
    rng = np.random.default_rng(0)
    for _ in range(50):
        f = rng.uniform(0, 20, 3).astype(np.float32)
        x = torch.from_numpy(f).double()
        h1 = torch.relu(w1.view(64, 3) @ x + b1)
        h2 = torch.relu(w2.view(64, 64) @ h1 + b2)
        want = float(w3 @ h2 + b3[0])
        got = O.mlp_logit(mlp, f.tolist())
        assert got == pytest.approx(want, rel=1e-4, abs=1e-4)


def _mlp32(seed):
    rng = np.random.default_rng(seed)
    return {"w1": rng.normal(0, 0.7, (64, 3)), "b1": rng.normal(0, 0.1, 64),
            "w2": rng.normal(0, 0.2, (64, 64)), "b2": rng.normal(0, 0.1, 64),
            "w3": rng.normal(0, 0.3, 64), "b3": np.array([0.05])}


def test_mlp_grad_matches_torch_autograd():
    w = _mlp32(1)
    rng = np.random.default_rng(2)
    feat = rng.uniform(0, 10, (300, 3)).astype(np.float32)
    label = (rng.uniform(size=300) < 0.3).astype(np.float32)
    loss, grads = O.mlp_loss_grad(w, feat, label)
    t = {k: torch.tensor(np.asarray(v, dtype=np.float32), dtype=torch.float64, requires_grad=True)
         for k, v in w.items()}
    x = torch.from_numpy(feat).double()
    h1 = torch.relu(x @ t["w1"].T + t["b1"])
    h2 = torch.relu(h1 @ t["w2"].T + t["b2"])
    z = h2 @ t["w3"] + t["b3"]
    tl = torch.nn.functional.binary_cross_entropy_with_logits(z, torch.from_numpy(label).double())
    tl.backward()
    assert loss == pytest.approx(float(tl), rel=1e-5)
    for k in w:
        np.testing.assert_allclose(grads[k], t[k].grad.numpy().reshape(grads[k].shape), rtol=2e-3, atol=2e-6)


def test_mlp_grad_finite_difference():
    w = _mlp32(4)
    rng = np.random.default_rng(5)
    feat = rng.uniform(0, 5, (64, 3)).astype(np.float32)
    label = (rng.uniform(size=64) < 0.5).astype(np.float32)
    _, grads = O.mlp_loss_grad(w, feat, label)
    h = 1e-2
    for name, idx in (("w1", (3, 1)), ("b2", (7,)), ("w2", (5, 9)), ("w3", (11,)), ("b3", (0,))):
        wp = {k: np.array(v, dtype=np.float64) for k, v in w.items()}
        wm = {k: np.array(v, dtype=np.float64) for k, v in w.items()}
        wp[name][idx] += h
        wm[name][idx] -= h
        fd = (O.mlp_loss_grad(wp, feat, label)[0] - O.mlp_loss_grad(wm, feat, label)[0]) / (2 * h)
        assert grads[name][idx] == pytest.approx(fd, rel=2e-2, abs=2e-4), name


def test_learned_large_sets_fall_back_to_uniform_and_stay_unbiased():
    """Candidate sets above 256 entries are drawn uniformly in learned mode;
    in K_300 the first candidate set of the 4-clique plan exceeds that bound
    for many first edges, so both kinds of steps occur, and the estimate is
    unbiased."""
    rp, col = G.complete(300)
    g = og(rp, col)
    p = O.plan(*G.pattern("4-clique"))
    mlp = random_mlp(5)
    _, recs = O.ns_run(g, p, seed=3, first=0, count=2000, mode=O.LEARNED, mlp=mlp, trace=True)
    sizes = recs["factor"][:, 2]
    learned = recs["aux"][:, 2] > 0
    uniform = (~learned) & (sizes > 0)
    assert learned.any() and uniform.any()
    assert np.all(sizes[uniform] > 256) and np.all(sizes[learned] > 0)
    # learned steps record A = sum of scores, each score in [1, 4097]
    assert np.all(recs["aux"][learned, 2] >= 1) and np.all(recs["aux"][learned, 2] <= 4097)
    N = 8_000
    acc, _ = O.ns_run(g, p, seed=4, first=0, count=N, mode=O.LEARNED, mlp=mlp)
    C = math.comb(300, 4)
    mean = acc.sum / N
    sd = math.sqrt(max(acc.sumsq / N - mean * mean, 0.0) / N)
    assert abs(mean - C) < 5 * sd + 1e-9 * C


# ------------------------------------------------------------------ NS-base (lazy verify)
def test_lazy_triangles_in_complete_graph_closed_form():
    """NS-base on K_n, triangle: the first edge is one of the n(n-1) directed
    entries, U_2 = N(v0) u N(v1) is every vertex (n of them), so every sample
    weighs n^2 (n-1), and a sample hits iff v0 < v1 < v2: C(n, 3) of the
    n^2 (n-1) equally likely paths.  The eager sampler misses only when the
    oriented first edge ends at the top vertex: n - 1 of the C(n, 2) edges."""
    n = 7
    rp, col = G.complete(n)
    g = og(rp, col)
    p = O.plan(*G.pattern("triangle"))
    W = n * n * (n - 1)
    leaves, total = enumerate_tree(g, p, O.LAZY)
    assert total == 1 and len(leaves) == math.comb(n, 3)
    for _, prob, rec in leaves:
        assert prob == Fraction(1, W) and rec.w_u64 == W
    N = 60_000
    acc, recs = O.ns_run(g, p, seed=3, first=0, count=N, mode=O.LAZY, trace=True)
    assert np.all(recs["factor"][:, 2] == n) and np.all(recs["factor"][:, 0] == n * (n - 1))
    q = math.comb(n, 3) / W
    assert abs(acc.hits / N - q) < 5 * math.sqrt(q * (1 - q) / N)
    eager, _ = O.ns_run(g, p, seed=3, first=0, count=N)
    qe = 1 - (n - 1) / math.comb(n, 2)
    assert abs(eager.hits / N - qe) < 5 * math.sqrt(qe * (1 - qe) / N)


def test_lazy_union_order_and_closure_on_a_path():
    """A 4-path graph 0-1-2-3 and the 4-cycle pattern (order 0-1-2-3: v2 from
    N(v1), v3 from N(v0) u N(v2)): from the first edge (1, 0), N(v1 = 0) = {1}
    gives v2 = 1, a repeated vertex the lazy sampler only rejects at the end;
    from (1, 2), N(2) = {1, 3} and U_3 = N(1) u N(3) = {0, 2} then {2} again:
    in list order 0, 2 (N(1) = {0, 2} first, N(3) = {2} adds nothing)."""
    rp, col = G.from_edge_list(4, [(0, 1), (1, 2), (2, 3)])
    g = og(rp, col)
    p = O.plan(*G.pattern("4-cycle"))
    assert list(p.order) [:4] == [0, 1, 2, 3]
    # directed entries: 0->1 (0), 1->0 (1), 1->2 (2), 2->1 (3), 2->3 (4), 3->2 (5)
    rec = O.sample(g, p, [_ceil_word(1, 6), 0, 0], mode=O.LAZY)
    assert rec.hit == 0 and rec.depth == 4 and [rec.vert[i] for i in range(3)] == [1, 0, 1]
    assert [rec.factor[j] for j in range(4)] == [6, 0, 1, 2]
    rec = O.sample(g, p, [_ceil_word(2, 6), _ceil_word(1, 2), _ceil_word(1, 2)], mode=O.LAZY)
    assert [rec.vert[i] for i in range(4)] == [1, 2, 3, 2] and rec.factor[3] == 2 and rec.hit == 0
    rec = O.sample(g, p, [_ceil_word(2, 6), _ceil_word(1, 2), _ceil_word(0, 2)], mode=O.LAZY)
    assert [rec.vert[i] for i in range(4)] == [1, 2, 3, 0] and rec.hit == 0    # 3-0 is not an edge


# ------------------------------------------------------------------ variance: sums against Welford
@pytest.mark.parametrize("name,induced,gen", [
    ("5-path", False, ("rmat", 12)),          # hit rate near 1: the smallest CV^2 of the workloads
    ("4-clique", False, ("rmat", 12)),
    ("triangle", False, ("er", 0)),
    ("wedge", False, ("complete", 9)),        # every sample hits with the same weight: var = 0
])
def test_sum_of_squares_variance_agrees_with_welford(name, induced, gen):
    """Algorithm 3 keeps sum X and sum X^2; var = sumsq / n - mu^2 cancels when
    CV^2 = var / mu^2 is small.  Its relative error is about
    eps_mach (1 + 1 / CV^2) n; Welford's update (M2 / n) does not cancel.  On the
    workloads' patterns the two agree within 1e-9 relative, and CV^2 stays far
    from the regime where they would not."""
    if gen[0] == "rmat":
        rp, col = G.rmat(gen[1], 16, seed=2)
    elif gen[0] == "er":
        rp, col = G.erdos_renyi(3000, 0.01, seed=2)
    else:
        rp, col = G.complete(gen[1])
    g = og(rp, col)
    k, edges = G.pattern(name)
    p = O.plan(k, edges, induced)
    N = 200_000
    acc, _ = O.ns_run(g, p, seed=3, first=0, count=N)
    mu_w, m2 = O.welford(g, p, seed=3, first=0, count=N)
    mu = acc.sum / N
    var_s = max(acc.sumsq / N - mu * mu, 0.0)
    var_w = m2 / N
    assert mu == pytest.approx(mu_w, rel=1e-12)
    if var_w == 0.0:
        assert var_s <= 1e-12 * mu * mu
        return
    cv2 = var_w / (mu_w * mu_w)
    assert abs(var_s - var_w) <= 1e-9 * var_w, (var_s, var_w, cv2)
    # the cancellation bound predicts this agreement: eps (1 + 1/CV^2) log2(N) is far below 1e-9
    assert 2.0 ** -52 * (1 + 1 / cv2) * math.log2(N) < 1e-9, cv2


# ------------------------------------------------------------------ GS variance model
def test_gs_variance_model_equals_the_variance_over_every_colouring():
    """The corrected variance model (oracle/gs_variance.py) against the exact
    variance of C' c^(k-1) over all c^n colourings of a small graph."""
    import itertools
    from oracle import gs_variance
    rp, col = G.random_small(8, 0.6, 31)
    rp_n, col_n = G.to_numpy(rp, col)
    g = og(rp, col)
    for name, c in (("triangle", 2), ("4-clique", 2), ("4-cycle", 3), ("wedge", 2)):
        k, edges = G.pattern(name)
        p = O.plan(k, edges)
        ms = brute.matches(rp_n, col_n, k, edges)
        C = len(ms)
        n = g.n
        if c ** n > 7000:
            continue
        s1 = s2 = Fraction(0)
        for cols in itertools.product(range(c), repeat=n):
            row, cc = O.sparsify(g, np.array(cols, dtype=np.uint32))
            x = Fraction(O.exact_count(O.Graph(row, cc), p) * c ** (k - 1))
            s1 += x
            s2 += x * x
        N = c ** n
        mean, var = s1 / N, s2 / N - (s1 / N) ** 2
        assert mean == C
        assert var == gs_variance.colour_variance(ms, k, c), name


def test_gs_edge_variance_model_equals_the_variance_over_every_edge_subset():
    """Bernoulli edge sparsification at p = 1/2: every subset of the m edges is
    equally likely; the variance of C' 2^l over all of them equals the model."""
    import itertools
    from oracle import gs_variance
    rp, col = G.random_small(7, 0.55, 12)
    rp_n, col_n = G.to_numpy(rp, col)
    edges_g = [(u, int(w)) for u in range(len(rp_n) - 1) for w in col_n[rp_n[u]:rp_n[u + 1]] if u < w]
    m = len(edges_g)
    assert m <= 14
    for name in ("triangle", "4-cycle", "wedge"):
        k, edges = G.pattern(name)
        p = O.plan(k, edges)
        ms = brute.matches(rp_n, col_n, k, edges)
        l = len(edges)
        s1 = s2 = Fraction(0)
        for keep in itertools.product((0, 1), repeat=m):
            kept = [e for e, b in zip(edges_g, keep) if b]
            rr, cc = G.to_numpy(*G.from_edge_list(len(rp_n) - 1, kept))
            x = Fraction(O.exact_count(O.Graph(rr, cc), p) * 2 ** l)
            s1 += x
            s2 += x * x
        N = 2 ** m
        assert s1 / N == len(ms)
        assert s2 / N - (s1 / N) ** 2 == gs_variance.edge_variance(ms, l, Fraction(1, 2)), name
