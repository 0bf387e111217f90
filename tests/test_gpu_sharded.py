"""Sharded rounds on one GPU with the ranks run one after another: each rank's
chunk partials (chunks dealt round robin), interleaved and merged on the host,
give gpm_sample_sums's totals bit for bit, and the sharded Algorithm 3 gives
gpm_estimate's result bit for bit."""
import pytest
import torch

from paper_2405_03488_gb300 import api, sharded
from paper_2405_03488_gb300 import graphs as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2405_03488_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


@pytest.fixture(scope="module")
def graph():
    rp, col = G.rmat(14, 16, seed=3, device="cuda")
    return api.Graph(rp, col)


@pytest.mark.parametrize("name", ["4-clique", "house", "4-cycle"])
@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_partials_merge_to_sample_sums(graph, name, world):
    first, count = 12_345, 100_003      # a ragged last chunk
    ref = graph.sample_sums(name, seed=4, first=first, count=count, slot=2)
    parts = [graph.sample_partials(name, 4, first, count, r, world, slot=2) for r in range(world)]
    assert sum(len(p) for p in parts) == (count + 63) // 64
    s = sharded.merge_partials(sharded.interleave(parts))
    assert (s.n, s.hits, s.sum, s.sumsq) == (ref.n, ref.hits, ref.sum, ref.sumsq)


def test_rank_without_chunks(graph):
    assert len(graph.sample_partials("triangle", 1, 0, 100, 3, 4)) == 0     # 2 chunks, rank 3 of 4
    assert len(graph.sample_partials("triangle", 1, 0, 0, 0, 1)) == 0


@pytest.mark.parametrize("name,world", [("4-clique", 2), ("5-clique", 3), ("4-cycle", 4)])
def test_sharded_estimate_equals_single_gpu(graph, name, world):
    seed, slot, W, eps = 21, 1, 1 << 14, 0.02
    last = {}

    def partials_fn(first, count, rank, w):
        last["fc"] = (first, count)
        return graph.sample_partials(name, seed, first, count, rank, w, slot=slot)

    def gather(local):
        first, count = last["fc"]
        return [local] + [graph.sample_partials(name, seed, first, count, r, world, slot=slot)
                          for r in range(1, world)]

    res = sharded.estimate_sharded(partials_fn, eps, 0.01, W, 0, world, gather)
    one = graph.estimate(name, eps=eps, delta=0.01, seed=seed, window=W, slot=slot)
    for f in ("estimate", "ci_half_width", "eps_hat", "samples", "hits", "rounds", "converged", "sum", "sumsq"):
        assert res[f] == one[f], f



def test_resumed_estimate_equals_single_gpu(graph):
    seed, W = 8, 1 << 14
    fn = lambda first, count, rank, world: graph.sample_partials("5-clique", seed, first, count, rank, world)
    gather = lambda local: [local]
    part = sharded.estimate_sharded(fn, 0.02, 0.01, W, 0, 1, gather, max_rounds=1)
    rest = sharded.estimate_sharded(fn, 0.02, 0.01, W, 0, 1, gather, state=bytes(part["state"]))
    one = graph.estimate("5-clique", eps=0.02, delta=0.01, seed=seed, window=W)
    assert one["rounds"] >= 2
    for f in ("estimate", "ci_half_width", "eps_hat", "samples", "hits", "rounds", "converged", "sum", "sumsq"):
        assert rest[f] == one[f], f
