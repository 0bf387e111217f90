"""Sharded rounds on one GPU.

Ranks run one after another, or as host threads that exchange their run sums
through a host barrier (their kernels never wait on one another): each rank's
run block (or round-robin chunk partials), gathered and folded on the host,
gives gpm_sample_sums's totals bit for bit, and the sharded Algorithm 3, in
Python or inside libgpm (gpm_estimate_sharded), gives gpm_estimate's result
bit for bit."""
import threading

import numpy as np
import pytest
import torch

from paper_2405_03488_gb300 import _lib, api, sharded
from paper_2405_03488_gb300 import graphs as G

pytestmark = pytest.mark.gpu

FIELDS = ("estimate", "ci_half_width", "eps_hat", "samples", "hits", "rounds", "converged", "sum", "sumsq")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2405_03488_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


@pytest.fixture(scope="module")
def rmat14():
    return G.rmat(14, 16, seed=3, device="cuda")


@pytest.fixture(scope="module")
def graph(rmat14):
    return api.Graph(*rmat14)


@pytest.mark.parametrize("name", ["4-clique", "house", "4-cycle"])
@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_partials_merge_to_sample_sums(graph, name, world):
    first, count = 12_345, 100_003      # a ragged last chunk
    ref = graph.sample_sums(name, seed=4, first=first, count=count, slot=2)
    parts = [graph.sample_partials(name, 4, first, count, r, world, slot=2) for r in range(world)]
    assert sum(len(p) for p in parts) == (count + 63) // 64
    s = sharded.merge_partials(sharded.interleave(parts))
    assert (s.n, s.hits, s.sum, s.sumsq) == (ref.n, ref.hits, ref.sum, ref.sumsq)


@pytest.mark.parametrize("name", ["4-clique", "house", "5-clique"])
@pytest.mark.parametrize("world", [1, 2, 3, 8, 1024])
def test_run_blocks_merge_to_sample_sums(graph, name, world):
    for first, count in ((12_345, 100_003), (0, 1 << 20), (7, 50)):
        ref = graph.sample_sums(name, seed=4, first=first, count=count, slot=2)
        runs = np.concatenate([graph.sample_runs(name, 4, first, count, r, world, slot=2) for r in range(world)])
        s = sharded.merge_runs(runs)
        assert (s.n, s.hits, s.sum, s.sumsq) == (ref.n, ref.hits, ref.sum, ref.sumsq)


def test_rank_without_chunks(graph):
    assert len(graph.sample_partials("triangle", 1, 0, 100, 3, 4)) == 0     # 2 chunks, rank 3 of 4
    assert len(graph.sample_partials("triangle", 1, 0, 0, 0, 1)) == 0
    runs = graph.sample_runs("triangle", 1, 0, 100, 3, 4)                   # 2 chunks: runs 0, 1 on rank 0
    assert len(runs) == 256 and runs["n"].sum() == 0


@pytest.mark.parametrize("name,world", [("4-clique", 2), ("5-clique", 3), ("4-cycle", 4)])
def test_python_sharded_estimate_equals_single_gpu(graph, name, world):
    seed, slot, W, eps = 21, 1, 1 << 14, 0.02
    last = {}

    def runs_fn(first, count, rank, w):
        last["fc"] = (first, count)
        return graph.sample_runs(name, seed, first, count, rank, w, slot=slot)

    def gather(local):
        first, count = last["fc"]
        return [local] + [graph.sample_runs(name, seed, first, count, r, world, slot=slot) for r in range(1, world)]

    res = sharded.estimate_sharded(runs_fn, eps, 0.01, W, 0, world, gather)
    one = graph.estimate(name, eps=eps, delta=0.01, seed=seed, window=W, slot=slot)
    for f in FIELDS:
        assert res[f] == one[f], f


class Exchange:
    """All-gather between host threads (one per rank) through two barriers."""

    def __init__(self, world):
        self.buf = [None] * world
        self.b1 = threading.Barrier(world, timeout=120)
        self.b2 = threading.Barrier(world, timeout=120)

    def gather_for(self, rank):
        def gather(block):
            self.buf[rank] = block
            self.b1.wait()
            out = np.concatenate(self.buf)
            self.b2.wait()
            return out
        return gather


@pytest.mark.parametrize("name,world,verify", [("4-clique", 2, "intersect"), ("5-clique", 3, "intersect"),
                                                ("4-cycle", 4, "check"), ("4-clique", 2, "lazy")])
def test_library_sharded_estimate_on_threads_equals_single_gpu(rmat14, graph, name, world, verify):
    """gpm_estimate_sharded with one host thread and one handle per rank."""
    seed, slot, W = 33, 2, 1 << 14
    eps = 0.1 if verify == "lazy" else 0.02
    handles = [api.Graph(*rmat14) for _ in range(world)]
    ex = Exchange(world)
    out = [None] * world
    errs = []

    def rank_main(r):
        try:
            out[r] = handles[r].estimate_sharded(name, r, world, ex.gather_for(r), eps=eps, delta=0.01, seed=seed,
                                                 window=W, slot=slot, verify=verify)
        except Exception as e:   # surfaced below
            errs.append(e)

    th = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs, errs
    one = graph.estimate(name, eps=eps, delta=0.01, seed=seed, window=W, slot=slot, verify=verify)
    assert one["converged"] == 1
    for r in range(world):
        for f in FIELDS:
            assert out[r][f] == one[f], (r, f)


def test_library_sharded_resume_and_failed_gather(graph):
    seed, W = 8, 1 << 14
    ident = lambda block: block
    st = _lib.Window()
    st.active = 1
    part = graph.estimate_sharded("5-clique", 0, 1, ident, eps=0.02, delta=0.01, seed=seed, window=W, state=st,
                                  max_rounds=1)
    assert part["rounds"] == 1 and st.active == 1 and st.rounds == 1
    rest = graph.estimate_sharded("5-clique", 0, 1, ident, eps=0.02, delta=0.01, seed=seed, window=W, state=st)
    one = graph.estimate("5-clique", eps=0.02, delta=0.01, seed=seed, window=W)
    assert one["rounds"] >= 2
    for f in FIELDS:
        assert rest[f] == one[f], f

    def broken(block):
        raise RuntimeError("peer lost")

    with pytest.raises(RuntimeError, match="peer lost"):
        graph.estimate_sharded("4-clique", 0, 2, broken, eps=0.02, window=W)
    r = graph.estimate("triangle", eps=0.05, delta=0.01, seed=2, window=W)    # the handle still works
    assert r["converged"] == 1
