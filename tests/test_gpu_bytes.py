"""The device's per-sample algorithmic byte count (gpm_sample_record.sectors,
trace mode) against the oracle's count on the same sample paths, and the mean
it reports in gpm_result.algo_bytes_per_sample.  The count is the graph data
the candidate-set definition of Sec. 4.2 references on the path a sample
takes; the oracle's count is pinned by hand in test_oracle_bytes.py."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2405_03488_gb300 import api
from paper_2405_03488_gb300 import graphs as G

pytestmark = pytest.mark.gpu

PATTERNS = [("triangle", False), ("4-clique", False), ("5-clique", False), ("4-cycle", False),
            ("4-cycle", True), ("diamond", False), ("tailed-triangle", True), ("3-star", True),
            ("house", False), ("5-path", True), ("wedge", True), ("dumbbell", False)]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2405_03488_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def bytes_gpu(g, pat, seed, first, count, **cfg):
    return 32.0 * g.trace(pat, seed=seed, first=first, count=count, **cfg)["sectors"].astype(np.float64)


@pytest.mark.parametrize("verify", ["intersect", "check", "lazy"])
@pytest.mark.parametrize("name,induced", PATTERNS)
def test_sectors_equal_oracle_small(name, induced, verify):
    rp, col = G.erdos_renyi(60, 0.25, seed=8)
    g = api.Graph(rp.cuda(), col.cuda())
    og = O.Graph(*G.to_numpy(rp, col))
    k, edges = G.pattern(name)
    mode = {"intersect": O.INTERSECT, "check": O.CHECK, "lazy": O.LAZY}[verify]
    gb = bytes_gpu(g, (k, edges, induced), 21, 777, 2500, verify=verify)
    cb = O.ns_bytes(og, O.plan(k, edges, induced), seed=21, first=777, count=2500, mode=mode)
    bad = np.nonzero(gb != cb)[0]
    assert len(bad) == 0, (bad[:5], gb[bad[:5]], cb[bad[:5]])


def test_sectors_equal_oracle_learned():
    rp, col = G.erdos_renyi(60, 0.25, seed=8)
    g = api.Graph(rp.cuda(), col.cuda())
    og = O.Graph(*G.to_numpy(rp, col))
    prop = api.Proposal(seed=4)
    gb = bytes_gpu(g, "4-clique", 5, 0, 2000, mlp=prop)
    cb = O.ns_bytes(og, O.plan(*G.pattern("4-clique")), seed=5, first=0, count=2000, mode=O.LEARNED,
                    mlp=O.Weights16(*prop.arrays16()))
    assert np.array_equal(gb, cb)


@pytest.fixture(scope="module")
def rmat22():
    rp, col = G.rmat(22, 16, seed=2, device="cuda")
    return rp, col


@pytest.mark.parametrize("name", ["4-clique", "5-clique", "4-cycle"])
def test_sectors_equal_oracle_rmat22(rmat22, name):
    """R-MAT scale 22, the benchmark's roofline workload, at two depths of the stream."""
    rp, col = rmat22
    g = api.Graph(rp, col)
    og = O.Graph(*G.to_numpy(rp, col))
    p = O.plan(*G.pattern(name))
    for first in (0, 987_654_321):
        gb = bytes_gpu(g, name, 1, first, 8192)
        cb = O.ns_bytes(og, p, seed=1, first=first, count=8192)
        assert np.array_equal(gb, cb)


def test_result_reports_mean_bytes_of_each_job():
    rp, col = G.rmat(14, 16, seed=2)
    g = api.Graph(rp.cuda(), col.cuda())
    og = O.Graph(*G.to_numpy(rp, col))
    names = ["4-clique", "4-cycle"]
    res = g.estimate_batch(names, [0.05, 0.05], delta=0.01, seed=3, window=1 << 14, bytes_sample=4096)
    for slot, (name, r) in enumerate(zip(names, res)):
        cb = O.ns_bytes(og, O.plan(*G.pattern(name)), seed=3, first=0, count=4096, slot=slot)
        assert r["algo_bytes_per_sample"] == pytest.approx(cb.mean(), rel=1e-12)
    r = g.estimate("5-clique", eps=0.05, delta=0.01, seed=3, window=1 << 14)
    assert r["algo_bytes_per_sample"] == 0.0
