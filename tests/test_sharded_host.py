"""Host logic of sharded rounds (Algorithm 3 with each window split over
ranks): the chunk-order merge is the device's fixed-shape reduction, and so is
the fold of run sums that ranks owning contiguous run blocks produce; the
window test follows Eq. equ:error step by step; two gloo ranks that each take
a block of every window reproduce the oracle's one-process online run."""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from oracle import oracle as O
from paper_2405_03488_gb300 import _lib, api, sharded
from paper_2405_03488_gb300 import graphs as G


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2405_03488_gb300 import build
    build.build()


def random_partials(n, seed):
    rng = np.random.default_rng(seed)
    p = np.zeros(n, dtype=api.PARTIAL_DTYPE)
    p["sum"] = rng.random(n) * 10.0 ** rng.integers(-3, 9, n)
    p["sumsq"] = p["sum"] ** 2 * rng.random(n)
    p["hits"] = rng.integers(0, 65, n)
    p["n"] = 64
    return p


def tree_reference(p):
    """1024 contiguous runs of ceil(n / 1024) partials added left to right, then
    run t += run t + h for h = 512, ..., 1."""
    n = len(p)
    per = (n + 1023) // 1024
    s = [0.0] * 1024
    for t in range(1024):
        acc = 0.0
        for i in range(t * per, min(t * per + per, n)):
            acc += float(p["sum"][i])
        s[t] = acc
    h = 512
    while h:
        for t in range(h):
            s[t] += s[t + h]
        h >>= 1
    return s[0]


@pytest.mark.parametrize("n", [0, 1, 7, 1023, 1024, 1025, 4097, 20000])
def test_merge_is_the_fixed_shape_reduction(n):
    p = random_partials(n, seed=n)
    s = sharded.merge_partials(p)
    assert s.n == int(p["n"].sum()) and s.hits == int(p["hits"].sum())
    assert s.sum == tree_reference(p)
    exact = math.fsum(p["sum"].tolist())
    assert s.sum == pytest.approx(exact, rel=1e-12, abs=0.0)
    assert s.sumsq == pytest.approx(math.fsum(p["sumsq"].tolist()), rel=1e-12, abs=0.0)


@pytest.mark.parametrize("n", [1, 63, 1024, 1025, 5000, 16384])
def test_run_blocks_fold_to_the_chunk_order_reduction(n):
    """Every world size: the ranks' run sums, concatenated in rank order and
    folded, equal the chunk-order reduction of all partials bit for bit."""
    p = random_partials(n, seed=n + 7)
    ref = sharded.merge_partials(p)
    count = 64 * n
    for world in (1, 2, 3, 5, 8, 1000, 1024):
        runs = []
        for r in range(world):
            lo, hi = sharded.rank_samples(count, r, world)
            runs.append(sharded.runs_from_partials(p[lo // 64:(hi + 63) // 64], count, r, world))
        got = sharded.merge_runs(np.concatenate(runs))
        assert (got.n, got.hits, got.sum, got.sumsq) == (ref.n, ref.hits, ref.sum, ref.sumsq), world


def test_rank_blocks_tile_the_window():
    for count in (1, 64, 65, 1 << 20, 3_000_017):
        for world in (1, 2, 3, 7, 8, 1024):
            spans = [sharded.rank_samples(count, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == count
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            assert all(lo % 64 == 0 or lo == count for lo, _ in spans)   # ranks past the end are empty


def test_interleave_restores_chunk_order():
    p = random_partials(1001, seed=3)
    for world in (1, 2, 3, 7):
        ranks = [p[r::world] for r in range(world)]
        assert np.array_equal(sharded.interleave(ranks), p)


def window_reference(sum_, sumsq, n, z):
    mu = sum_ / n
    var = sumsq / n - mu * mu
    var = max(var, 0.0)
    sigma = math.sqrt(var / n)
    half = z * sigma
    return mu, half, (half / mu if mu > 0 else math.inf)


def test_window_update_follows_the_window_test():
    z = _lib.load().gpm_normal_quantile(1 - 0.01 / 2)
    assert z == pytest.approx(2.5758293035489004, rel=1e-15)
    st = _lib.Window()
    st.active = 1
    rng = np.random.default_rng(5)
    tot_s = tot_q = 0.0
    tot_n = tot_h = 0
    for r in range(6):
        w = _lib.Sums()
        w.n, w.hits = 4096, int(rng.integers(100, 4096))
        w.sum = float(rng.random() * 1e9)
        w.sumsq = float(w.sum ** 2 / 50 * (1 + rng.random()))
        sharded.window_update(st, w, z, 1e-9, 4096, 1 << 40)
        tot_s = w.sum if r == 0 else tot_s + w.sum
        tot_q = w.sumsq if r == 0 else tot_q + w.sumsq
        tot_n += w.n
        tot_h += w.hits
        mu, half, eh = window_reference(tot_s, tot_q, tot_n, z)
        assert (st.sum, st.sumsq, st.n, st.hits, st.rounds) == (tot_s, tot_q, tot_n, tot_h, r + 1)
        assert (st.mu, st.half, st.eps_hat) == (mu, half, eh)
        assert st.active == 1 and st.converged == 0
    # eps_hat = z sigma / mu on the sample: population variance over n (Eq. equ:error)
    x = np.array([0.0, 3.0, 0.0, 5.0, 4.0, 0.0, 0.0, 8.0])
    st2 = _lib.Window()
    st2.active = 1
    w = _lib.Sums()
    w.n, w.hits, w.sum, w.sumsq = len(x), 4, float(x.sum()), float((x * x).sum())
    sharded.window_update(st2, w, z, 10.0, 1, 100)
    assert st2.eps_hat == pytest.approx(z * x.std() / math.sqrt(len(x)) / x.mean(), rel=1e-14)
    assert st2.converged == 1 and st2.active == 0
    # no hits: mu = 0 never converges; n_max stops the run
    st3 = _lib.Window()
    st3.active = 1
    w0 = _lib.Sums()
    w0.n = 64
    sharded.window_update(st3, w0, z, 0.5, 64, 64)
    assert st3.converged == 0 and st3.active == 0 and math.isinf(st3.eps_hat)


SEED, SLOT, EPS, DELTA, W = 17, 3, 0.04, 0.01, 1 << 11


def oracle_partials(og, p, first, count, rank, world):
    nch = (count + 63) // 64
    mine = list(range(rank, nch, world))
    out = np.zeros(len(mine), dtype=api.PARTIAL_DTYPE)
    for i, c in enumerate(mine):
        s0 = first + 64 * c
        acc, _ = O.ns_run(og, p, seed=SEED, first=s0, count=min(64, first + count - s0), slot=SLOT)
        out[i] = (acc.sum, acc.sumsq, acc.hits, acc.n)
    return out


def oracle_runs(og, p, first, count, rank, world):
    """This rank's run sums, its block's chunk partials drawn by the oracle."""
    lo, hi = sharded.rank_samples(count, rank, world)
    parts = np.zeros((hi - lo + 63) // 64, dtype=api.PARTIAL_DTYPE)
    for i in range(len(parts)):
        s0 = first + lo + 64 * i
        acc, _ = O.ns_run(og, p, seed=SEED, first=s0, count=min(64, first + hi - s0), slot=SLOT)
        parts[i] = (acc.sum, acc.sumsq, acc.hits, acc.n)
    return sharded.runs_from_partials(parts, count, rank, world)


def _rank_main(rank, world, port, rp, col, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        og = O.Graph(rp, col)
        p = O.plan(*G.pattern("4-clique"))
        res = sharded.estimate_sharded(lambda f, c, r, w: oracle_runs(og, p, f, c, r, w), EPS, DELTA, W,
                                       rank, world, sharded.torch_gather())
        np.save(os.path.join(out_dir, "r%d.npy" % rank),
                np.array([res["estimate"], res["eps_hat"], res["samples"], res["hits"], res["rounds"],
                          res["converged"], res["sum"], res["sumsq"]], dtype=np.float64))
    finally:
        torch.distributed.destroy_process_group()


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reproduce_the_online_run(tmp_path):
    rp, col = G.to_numpy(*G.erdos_renyi(300, 0.08, seed=8))
    mp.spawn(_rank_main, args=(2, free_port(), rp, col, str(tmp_path)), nprocs=2, join=True)
    r0, r1 = (np.load(os.path.join(tmp_path, "r%d.npy" % r)) for r in (0, 1))
    assert np.array_equal(r0, r1)          # every rank reaches the same decision and totals
    og = O.Graph(rp, col)
    o = O.ns_online(og, O.plan(*G.pattern("4-clique")), EPS, DELTA, seed=SEED, window=W, slot=SLOT)
    assert o.converged == 1 and r0[5] == 1
    assert (r0[2], r0[3], r0[4]) == (o.samples, o.hits, o.rounds)
    assert r0[0] == pytest.approx(o.estimate, rel=1e-12)
    assert r0[1] == pytest.approx(o.eps_hat, rel=1e-10)
    # one process, same chunk partials, merged the same way: identical bits
    one = sharded.estimate_sharded(lambda f, c, r, w: oracle_runs(og, O.plan(*G.pattern("4-clique")), f, c, r, w),
                                   EPS, DELTA, W, 0, 1, lambda local: [local])
    assert (one["estimate"], one["sum"], one["sumsq"]) == (r0[0], r0[6], r0[7])


def test_checkpoint_and_resume_equal_the_uninterrupted_run():
    """Stopping after two windows, saving the 72-byte window state and resuming
    from it gives the uninterrupted run's result bit for bit (the sample streams
    are counter-based, so window r is the same samples either way)."""
    rp, col = G.to_numpy(*G.erdos_renyi(300, 0.08, seed=8))
    og = O.Graph(rp, col)
    p = O.plan(*G.pattern("4-clique"))
    fn = lambda f, c, r, w: oracle_runs(og, p, f, c, r, w)
    gather = lambda local: [local]
    full = sharded.estimate_sharded(fn, EPS, DELTA, W, 0, 1, gather)
    assert full["converged"] == 1 and full["rounds"] >= 3
    part = sharded.estimate_sharded(fn, EPS, DELTA, W, 0, 1, gather, max_rounds=2)
    assert part["active"] == 1 and part["rounds"] == 2
    saved = bytes(part["state"])
    assert len(saved) == 72
    rest = sharded.estimate_sharded(fn, EPS, DELTA, W, 0, 1, gather, state=saved)
    for f in ("estimate", "ci_half_width", "eps_hat", "samples", "hits", "rounds", "converged", "sum", "sumsq"):
        assert rest[f] == full[f], f


def masked_colours(n, c, seed, rank, world):
    """Colours with every class c != rank (mod world) replaced by one colour per
    vertex, so only the rank's classes keep edges."""
    cols = O.colors(n, c, seed).astype(np.uint64)
    v = np.arange(n, dtype=np.uint64)
    return np.where(cols % world == rank, cols, np.uint64(0xFFFFFFFF) - v).astype(np.uint32)


def _gs_rank_main(rank, world, port, rp, col, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        og = O.Graph(rp, col)
        k, edges = G.pattern("4-clique")
        p = O.plan(k, edges)

        def count_fn(r, w):
            row, cc = O.sparsify(og, masked_colours(og.n, 4, 23, r, w))
            return O.exact_count(O.Graph(row, cc), p)

        res = sharded.gs_estimate_sharded(count_fn, 4, k, rank, world, sharded.torch_allreduce_sum())
        np.save(os.path.join(out_dir, "g%d.npy" % rank), np.array([res["exact_count"], res["estimate"]]))
    finally:
        torch.distributed.destroy_process_group()


def test_two_gloo_ranks_split_gs_by_colour_class(tmp_path):
    """Sharded GS: each rank counts the matches of its colour classes; the
    integer all-reduce equals the count on the whole sparsified graph."""
    rp, col = G.to_numpy(*G.erdos_renyi(400, 0.12, seed=9))
    mp.spawn(_gs_rank_main, args=(2, free_port(), rp, col, str(tmp_path)), nprocs=2, join=True)
    g0, g1 = (np.load(os.path.join(tmp_path, "g%d.npy" % r)) for r in (0, 1))
    assert np.array_equal(g0, g1)
    og = O.Graph(rp, col)
    k, edges = G.pattern("4-clique")
    est, cp = O.gs_estimate(og, O.plan(k, edges), 4, seed=23)
    assert cp > 0 and g0[0] == cp and g0[1] == est
