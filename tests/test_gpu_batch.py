"""Batched persistent launches with graph-captured convergence rounds: every
job of a batch equals its separate single-pattern run bit for bit and the
oracle's online run within FP64 reduction order; results do not depend on the
launch shape; the autotuner returns a valid shape."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2405_03488_gb300 import api
from paper_2405_03488_gb300 import graphs as G

pytestmark = pytest.mark.gpu

REL = 1e-12
FIELDS = ("estimate", "eps_hat", "ci_half_width", "samples", "hits", "rounds", "converged", "sum", "sumsq")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2405_03488_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


@pytest.fixture(scope="module")
def rmat14():
    rp, col = G.rmat(14, 16, seed=3, device="cpu")
    return rp, col


def motif_jobs():
    names = G.MOTIFS4 + ["triangle"]
    pats, eps = [], []
    for e in (0.02, 0.05, 0.1):
        for nm in names:
            k, edges = G.pattern(nm)
            pats.append((k, edges, nm != "triangle"))     # 4-vertex motifs are vertex-induced
            eps.append(e)
    return pats, eps


def test_batch_equals_single_runs_and_oracle(rmat14):
    rp, col = rmat14
    g = api.Graph(rp.cuda(), col.cuda())
    og = O.Graph(*G.to_numpy(rp, col))
    pats, eps = motif_jobs()
    W = 1 << 14
    res = g.estimate_batch(pats, eps, delta=0.01, seed=5, window=W, n_max=1 << 22)
    assert len(res) == 21
    again = g.estimate_batch(pats, eps, delta=0.01, seed=5, window=W, n_max=1 << 22)
    for a, b in zip(res, again):      # run-to-run: the fixed chunk-order reduction is deterministic
        for f in FIELDS:
            assert a[f] == b[f], f
    for q, (pat, e) in enumerate(zip(pats, eps)):
        single = g.estimate(pat, eps=e, delta=0.01, seed=5, window=W, n_max=1 << 22, slot=q)
        for f in FIELDS:
            assert res[q][f] == single[f], (q, f)
    # a few jobs against the oracle's online run on the same slot
    for q in (0, 3, 6, 13, 20):
        k, edges, induced = pats[q]
        o = O.ns_online(og, O.plan(k, edges, induced), eps[q], 0.01, seed=5, window=W, n_max=1 << 22, slot=q)
        assert res[q]["samples"] == o.samples and res[q]["hits"] == o.hits and res[q]["converged"] == o.converged
        assert res[q]["estimate"] == pytest.approx(o.estimate, rel=REL)
        assert res[q]["eps_hat"] == pytest.approx(o.eps_hat, rel=1e-10)


@pytest.mark.parametrize("warps,cap,blocks", [(2, 256, 0), (4, 1024, 0), (8, 64, 37), (1, 16, 5)])
def test_results_do_not_depend_on_launch_shape(rmat14, warps, cap, blocks):
    rp, col = rmat14
    g = api.Graph(rp.cuda(), col.cuda())
    pats = ["4-clique", "4-cycle", "5-clique"]
    ref = g.estimate_batch(pats, [0.03] * 3, seed=9, window=1 << 14)
    got = g.estimate_batch(pats, [0.03] * 3, seed=9, window=1 << 14, block_warps=warps, cap=cap,
                           grid_blocks=blocks)
    for a, b in zip(ref, got):
        for f in FIELDS:
            assert a[f] == b[f], f


def test_batch_check_mode_and_unconverged(rmat14):
    rp, col = rmat14
    g = api.Graph(rp.cuda(), col.cuda())
    og = O.Graph(*G.to_numpy(rp, col))
    res = g.estimate_batch(["4-clique", "triangle"], [1e-6, 0.05], seed=2, window=1 << 13, n_max=1 << 15,
                           verify="check")
    assert res[0]["converged"] == 0 and res[0]["samples"] == 1 << 15
    assert res[1]["converged"] == 1
    o = O.ns_online(og, O.plan(*G.pattern("triangle")), 0.05, 0.01, seed=2, window=1 << 13, n_max=1 << 15,
                    mode=O.CHECK, slot=1)
    assert res[1]["samples"] == o.samples and res[1]["estimate"] == pytest.approx(o.estimate, rel=REL)


def test_autotune_returns_a_valid_shape(rmat14):
    rp, col = rmat14
    g = api.Graph(rp.cuda(), col.cuda())
    best = g.autotune(["4-clique", "5-clique"], window=1 << 14)
    assert best["block_warps"] in (4, 8)
    assert best["cap"] in (256, 512) or (best["cap"] >= 512 and best["cap"] % 32 == 0)
    r = g.estimate("4-clique", eps=0.05, seed=1, window=1 << 14, **best)
    assert r["converged"] == 1


def test_mixed_batch_runs_single_list_variant_bit_exact(rmat14):
    """A batch with edge-induced paths and cycles runs the sampler variant that
    evaluates one-list steps by positions; every job, the cliques included,
    still equals its separate run and the oracle."""
    rp, col = rmat14
    g = api.Graph(rp.cuda(), col.cuda())
    og = O.Graph(*G.to_numpy(rp, col))
    names = ["4-clique", "4-cycle", "5-path", "house", "wedge", "5-clique"]
    W = 1 << 14
    res = g.estimate_batch(names, [0.02] * len(names), seed=4, window=W, n_max=1 << 22)
    for q, nm in enumerate(names):
        single = g.estimate(nm, eps=0.02, seed=4, window=W, n_max=1 << 22, slot=q)
        for f in FIELDS:
            assert res[q][f] == single[f], (nm, f)
    for q in (1, 2):
        k, edges = G.pattern(names[q])
        o = O.ns_online(og, O.plan(k, edges, False), 0.02, 0.01, seed=4, window=W, n_max=1 << 22, slot=q)
        assert res[q]["samples"] == o.samples and res[q]["hits"] == o.hits
        assert res[q]["estimate"] == pytest.approx(o.estimate, rel=REL)
