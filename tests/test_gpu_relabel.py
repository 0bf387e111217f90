"""GPM_RELABEL_DEGREE: the library relabels a loaded CSR by (degree, id) on the
device (the clique orientation of Table tab:input's caption, as this library
reads it).  The relabelled graph must be exactly the one the CPU relabelling
of the input generator gives, so 4-clique records on it equal the oracle's on
that graph bit for bit."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2405_03488_gb300 import _lib, api
from paper_2405_03488_gb300 import graphs as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2405_03488_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def expected_map(rp):
    deg = (rp[1:] - rp[:-1]).to(torch.int64)
    order = torch.sort(deg, stable=True).indices
    newid = torch.empty_like(order)
    newid[order] = torch.arange(len(order))
    return newid.numpy().astype(np.uint32)


@pytest.mark.parametrize("device_ptrs", [True, False])
def test_relabelled_rmat14_records_equal_oracle(device_ptrs):
    rp, col = G.rmat(14, 16, seed=6, relabel=False)
    g = api.Graph(rp.cuda(), col.cuda(), relabel=True) if device_ptrs else \
        api.Graph(rp.numpy(), col.numpy(), relabel=True)
    assert np.array_equal(g.relabel_map(), expected_map(rp))
    rrp, rcol = G.relabel_by_degree(rp, col)
    og = O.Graph(*G.to_numpy(rrp, rcol))
    assert (g.n, g.nnz) == (og.n, og.nnz) and g.m == og.m
    for name in ("4-clique", "4-cycle"):
        k, edges = G.pattern(name)
        gpu = g.trace(name, seed=3, first=1000, count=20_000)
        _, cpu = O.ns_run(og, O.plan(k, edges), seed=3, first=1000, count=20_000, trace=True)
        for f in ("hit", "depth", "w_u64"):
            assert np.array_equal(gpu[f], cpu[f]), (name, f)
        assert np.array_equal(gpu["vert"][:, :k], cpu["vert"][:, :k])
        assert np.array_equal(gpu["w_f64"].view(np.uint64), cpu["w_f64"].view(np.uint64))
    assert g.exact_count("4-clique") == O.exact_count(og, O.plan(*G.pattern("4-clique")))


def test_relabel_small_and_degenerate_graphs():
    # isolated vertices, ties in degree, a single vertex, no edges
    rp, col = G.from_edge_list(9, [(0, 5), (5, 7), (7, 0), (2, 3), (8, 5)])
    g = api.Graph(rp.cuda(), col.cuda(), relabel=True, validate=True)
    m = g.relabel_map()
    assert np.array_equal(m, expected_map(rp))
    rrp, rcol = G.relabel_by_degree(rp, col)
    assert g.exact_count("triangle") == 1
    tr = g.trace("edge", seed=1, first=0, count=64)
    assert set(map(int, tr["vert"][:, 0])) <= set(range(9))
    for n in (1, 3):
        rp0, col0 = G.from_edge_list(n, [])
        g0 = api.Graph(rp0.cuda(), col0.cuda(), relabel=True)
        assert np.array_equal(g0.relabel_map(), np.arange(n, dtype=np.uint32))
    g1 = api.Graph(rp.cuda(), col.cuda())
    with pytest.raises(_lib.GpmError):
        g1.relabel_map()
