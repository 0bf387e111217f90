"""The synthetic inputs every parity test and benchmark runs on: generated
graphs are valid symmetric CSRs (sorted, deduplicated, loop-free), seeded and
reproducible, degree-relabelled when asked; the partitioned deduplication that
billion-edge graphs take gives the same graph as a single pass; G(n, p) and
the planted cliques have the expected counts."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2405_03488_gb300 import graphs as G


def valid(rp, col):
    return O.validate(*G.to_numpy(rp, col)) == 0


def test_rmat_is_valid_seeded_and_degree_ordered():
    rp, col = G.rmat(12, 16, seed=3)
    assert valid(rp, col)
    rp2, col2 = G.rmat(12, 16, seed=3)
    assert torch.equal(rp, rp2) and torch.equal(col, col2)
    rp3, col3 = G.rmat(12, 16, seed=4)
    assert not (rp.shape == rp3.shape and torch.equal(rp, rp3) and torch.equal(col, col3))
    deg = (rp[1:] - rp[:-1]).numpy()
    assert np.all(np.diff(deg) >= 0)             # relabelled by (degree, id)
    assert (deg > 0).sum() > 0.5 * len(deg) and rp[-1] <= 2 * 16 * (1 << 12)
    rpu, colu = G.rmat(12, 16, seed=3, relabel=False)
    assert valid(rpu, colu) and rpu[-1] == rp[-1]


def test_partitioned_deduplication_matches_one_pass(monkeypatch):
    """Above the sort library's size limit the keys are deduplicated in parts
    split at source vertices; forcing that path on a small graph gives the
    same CSR as one pass."""
    one = G.rmat(11, 16, seed=5)
    monkeypatch.setattr(G, "_UNIQUE_LIMIT", 5000)
    parts = G.rmat(11, 16, seed=5)
    assert torch.equal(one[0], parts[0]) and torch.equal(one[1], parts[1])
    assert valid(*parts)


def test_erdos_renyi_edge_count():
    n, p = 3000, 0.004
    rp, col = G.erdos_renyi(n, p, seed=11)
    assert valid(rp, col)
    m = int(rp[-1]) // 2
    mean = n * (n - 1) / 2 * p
    assert abs(m - mean) < 5 * math.sqrt(mean * (1 - p))


@pytest.mark.parametrize("k,planted", [(6, 4), (7, 3)])
def test_chung_lu_contains_the_planted_cliques(k, planted):
    """The background edges are drawn before the cliques from the same seeded
    generator, so planting adds each planted 12-vertex clique's C(12, k)
    k-cliques to the background's count (cliques of uniformly chosen vertices
    almost never share k vertices with each other or with a background clique)."""
    kk, edges = G.clique(k)
    counts = []
    for n_cliques in (0, planted):
        rp, col = G.chung_lu(3000, n_cliques=n_cliques, clique_size=12, seed=6)
        assert valid(rp, col)
        counts.append(O.exact_count(O.Graph(*G.to_numpy(rp, col)), O.plan(kk, edges)))
    assert counts[1] - counts[0] >= 0.99 * planted * math.comb(12, k)
