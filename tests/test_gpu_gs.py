"""GPU parity of colour sparsification, exact counting, the GS estimate and
the hybrid choice against the CPU oracle (integers bit-exact)."""
import math

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


def pair(rp, col):
    return api.Graph(rp.cuda(), col.cuda(), validate=True), O.Graph(*G.to_numpy(rp, col))


@pytest.mark.parametrize("c,colouring,slot", [(1, 0, 0), (2, 0, 0), (8, 3, 1), (1000, 1, 5)])
def test_sparsify_bit_exact(c, colouring, slot):
    rp, col = G.erdos_renyi(5000, 0.004, seed=6)
    g, og = pair(rp, col)
    row_d, col_d = g.sparsify(c, seed=99, colouring=colouring, slot=slot)
    cols = O.colors(og.n, c, 99, colouring, slot)
    row_o, col_o = O.sparsify(og, cols)
    assert np.array_equal(row_d.cpu().numpy().astype(np.uint64), row_o)
    assert np.array_equal(col_d.cpu().numpy().astype(np.uint32), col_o)


EXACT_PATTERNS = [("triangle", False), ("4-clique", False), ("5-clique", False), ("4-cycle", False),
                  ("4-cycle", True), ("diamond", True), ("house", False), ("3-star", True), ("4-path", True),
                  ("tailed-triangle", False), ("5-path", False), ("edge", False)]


@pytest.mark.parametrize("name,induced", EXACT_PATTERNS)
def test_exact_count_matches_oracle(name, induced):
    k, edges = G.pattern(name)
    for rp, col in (G.erdos_renyi(60, 0.25, seed=1), G.erdos_renyi(400, 0.03, seed=2), G.complete(9)):
        g, og = pair(rp, col)
        assert g.exact_count((k, edges, induced)) == O.exact_count(og, O.plan(k, edges, induced))


def test_exact_scheme_and_closed_forms():
    for n in (12, 20):
        rp, col = G.complete(n)
        g = api.Graph(rp.cuda(), col.cuda())
        for k in (3, 4, 5, 6):
            r = g.estimate("%d-clique" % k, scheme=api.EXACT)
            import math
            assert r["exact_count"] == math.comb(n, k) and r["estimate"] == math.comb(n, k)


@pytest.mark.parametrize("name,c", [("triangle", 2), ("4-clique", 4), ("4-cycle", 8), ("house", 3)])
def test_gs_estimate_matches_oracle(name, c):
    rp, col = G.erdos_renyi(3000, 0.01, seed=3)
    g, og = pair(rp, col)
    k, edges = G.pattern(name)
    r = g.estimate(name, scheme=api.GS, seed=17, colors=c)
    est, cp = O.gs_estimate(og, O.plan(k, edges), c, seed=17)
    assert r["scheme_used"] == api.GS
    assert r["exact_count"] == cp
    assert r["estimate"] == est
    assert np.isnan(r["ci_half_width"])


def test_hybrid_returns_a_consistent_engine_result():
    # dense-ish ER: NS converges quickly; planted cliques in a sparse graph: needle case
    rp, col = G.erdos_renyi(3000, 0.01, seed=4)
    g, og = pair(rp, col)
    r = g.estimate("triangle", scheme=api.HYBRID, eps=0.05, delta=0.01, seed=3, window=1 << 16)
    assert r["scheme_used"] in (api.NS, api.GS) and r["t_pilot_s"] > 0
    check_engine_result(r, og, "triangle", 8)
    rp, col = G.chung_lu(20000, n_cliques=20, clique_size=10, seed=5)
    g, og = pair(rp, col)
    r = g.estimate("6-clique", scheme=api.HYBRID, eps=0.05, delta=0.01, seed=3, window=1 << 16,
                   n_max=1 << 22, colors=2)
    check_engine_result(r, og, "6-clique", 2)


def test_hybrid_never_picks_gs_that_cannot_meet_the_target():
    """A few planted cliques in a sparse graph: with c = 8 colours a 6-clique
    survives with probability 8^-5, so GS's relative error is at least
    z sqrt((8^5 - 1) / C), far above eps; the hybrid must run NS."""
    rp, col = G.chung_lu(20000, n_cliques=20, clique_size=10, seed=5)
    g = api.Graph(rp.cuda(), col.cuda())
    C = g.exact_count("6-clique")
    z = api.normal_quantile(1.0 - 0.01 / 2)
    assert z * math.sqrt((8.0 ** 5 - 1.0) / C) > 0.05
    info = g.hybrid_model("6-clique", eps=0.05, delta=0.01, seed=3, window=1 << 16, colors=8)
    assert info["cost_model_gs"] == 0
    r = g.estimate("6-clique", scheme=api.HYBRID, eps=0.05, delta=0.01, seed=3, window=1 << 16, n_max=1 << 22,
                   colors=8)
    assert r["scheme_used"] == api.NS


def check_engine_result(r, og, name, colors):
    """Whichever engine the hybrid chose, its result is that engine's own: the
    oracle's online NS run (same seed and window) or its GS estimate."""
    k, edges = G.pattern(name)
    assert r["scheme_used"] in (api.NS, api.GS) and r["t_pilot_s"] > 0
    if r["scheme_used"] == api.NS:
        o = O.ns_online(og, O.plan(k, edges), 0.05, 0.01, seed=3, window=1 << 16, n_max=1 << 22)
        assert r["converged"] == o.converged
        assert (r["samples"], r["hits"], r["rounds"]) == (o.samples, o.hits, o.rounds)
        assert r["estimate"] == pytest.approx(o.estimate, rel=1e-12)
        assert r["eps_hat"] == pytest.approx(o.eps_hat, rel=1e-10)
    else:
        est, _ = O.gs_estimate(og, O.plan(k, edges), colors, seed=3)
        assert r["estimate"] == est


def test_exact_count_deadline_returns_a_lower_bound():
    """max_seconds bounds the exact search on the device: the 7-cliques of K_200
    (about 2.2e12) cannot be enumerated in 0.2 s, so the call returns
    NOT_CONVERGED with a partial count instead of running on."""
    import math
    import time
    rp, col = G.complete(200)
    g = api.Graph(rp.cuda(), col.cuda())
    t0 = time.perf_counter()
    r = g.estimate("7-clique", scheme=api.EXACT, max_seconds=0.2)
    dt = time.perf_counter() - t0
    assert r["status"] == -5 and r["converged"] == 0
    assert 0 < r["exact_count"] < math.comb(200, 7)
    assert dt < 5.0
    # a small case finishes inside the budget and is exact
    r = g.estimate("triangle", scheme=api.EXACT, max_seconds=30.0)
    assert r["converged"] == 1 and r["exact_count"] == math.comb(200, 3)


def test_selector_head_decides_the_hybrid():
    """A selector head trained on a few cases decides the hybrid's choice from
    the features of that very call, and the hybrid returns that engine's result."""
    import torch
    rp, col = G.erdos_renyi(3000, 0.01, seed=4)
    g = api.Graph(rp.cuda(), col.cuda())
    feats, labels = [], []
    for name in ("triangle", "4-clique", "4-cycle", "house"):
        info = g.hybrid_model(name, eps=0.05, delta=0.01, seed=3, window=1 << 15)
        assert len(info["features"]) == 3 and info["selector_gs"] == -1
        assert info["cost_model_gs"] in (0, 1) and info["t_lo"] <= info["t_hi"]
        feats.append(info["features"])
        labels.append(float(info["cost_model_gs"] == 0))   # train the head to disagree with the cost model
    sel = api.Proposal(seed=5)
    loss = sel.train_rows(g, torch.tensor(feats).cuda(), torch.tensor(labels).cuda(), epochs=500, batch=8, lr=2e-2)
    assert np.isfinite(loss)
    for name in ("triangle", "4-clique", "4-cycle", "house"):
        # the features include measured times, so compare against this call's own features
        info = g.hybrid_model(name, eps=0.05, delta=0.01, seed=3, window=1 << 15, selector=sel)
        want = int(sel.scores(g, torch.tensor([info["features"]]).cuda())[0].item() >= 2049)
        assert info["selector_gs"] == want
        r = g.estimate(name, scheme=api.HYBRID, eps=0.05, delta=0.01, seed=3, window=1 << 15, selector=sel)
        assert r["scheme_used"] in (api.NS, api.GS)
        if r["scheme_used"] == api.GS:
            assert r["estimate"] == g.estimate(name, scheme=api.GS, seed=3)["estimate"]
        else:
            assert r["converged"] == 1


@pytest.mark.parametrize("prob,colouring,slot", [(0.5, 0, 0), (0.3, 2, 1), (1.0, 0, 3), (0.05, 7, 0)])
def test_edge_sparsify_bit_exact(prob, colouring, slot):
    rp, col = G.erdos_renyi(5000, 0.004, seed=6)
    g, og = pair(rp, col)
    row_d, col_d = g.sparsify_edges(prob, seed=99, colouring=colouring, slot=slot)
    row_o, col_o = O.bes_sparsify(og, 99, O.bes_threshold(prob), colouring, slot)
    assert np.array_equal(row_d.cpu().numpy().astype(np.uint64), row_o)
    assert np.array_equal(col_d.cpu().numpy().astype(np.uint32), col_o)


def scaled_counts(og, name, seed, R, prob=None, c=None):
    """Per-sampler scaled counts from the oracle: sparsification r, exact count, scale."""
    k, edges = G.pattern(name)
    p = O.plan(k, edges)
    out = []
    for r in range(R):
        if prob is not None:
            t = O.bes_threshold(prob)
            row, cc = O.bes_sparsify(og, seed, t, colouring=r)
            scale = 1.0
            for _ in range(len(edges)):
                scale *= 4294967296.0 / t
        else:
            row, cc = O.sparsify(og, O.colors(og.n, c, seed, colouring=r))
            scale = float(c) ** (k - 1)
        out.append((O.exact_count(O.Graph(row, cc), p), scale))
    return out


@pytest.mark.parametrize("name,prob,c,R", [("triangle", 0.5, None, 1), ("4-cycle", 0.6, None, 5),
                                           ("house", 0.7, None, 3), ("4-clique", None, 4, 6)])
def test_gs_samplers_and_edge_mode_match_oracle(name, prob, c, R):
    rp, col = G.erdos_renyi(2000, 0.03, seed=7)
    g, og = pair(rp, col)
    kw = {"samplers": R}
    if prob is not None:
        kw["edge_p"] = prob
    else:
        kw["colors"] = c
    r = g.estimate(name, scheme=api.GS, seed=11, delta=0.05, **kw)
    parts = scaled_counts(og, name, 11, R, prob, c)
    ests = [cnt * s for cnt, s in parts]
    mean = 0.0
    for e in ests:
        mean += e
    mean /= R
    assert r["exact_count"] == sum(cnt for cnt, _ in parts)
    assert r["estimate"] == mean and r["samples"] == R
    if R == 1:
        assert np.isnan(r["ci_half_width"])
    else:
        ss = 0.0
        for e in ests:
            ss += (e - mean) * (e - mean)
        half = api.normal_quantile(1 - 0.05 / 2) * (math.sqrt(ss / (R - 1)) / math.sqrt(R))
        assert mean > 0
        assert r["ci_half_width"] == half and r["eps_hat"] == half / mean


def test_gs_edge_mode_refuses_vertex_induced_patterns():
    rp, col = G.erdos_renyi(300, 0.05, seed=2)
    g = api.Graph(rp.cuda(), col.cuda())
    k, edges = G.pattern("4-cycle")
    with pytest.raises(_lib.GpmError):
        g.estimate((k, edges, True), scheme=api.GS, edge_p=0.5)


@pytest.mark.parametrize("world", [1, 2, 3])
def test_gs_counts_by_colour_class_add_up(world):
    """The multi-GPU form of GS with the ranks run one after another: each
    rank's class count equals the oracle's on the same classes, and the ranks
    add up to the unsharded GS count."""
    rp, col = G.erdos_renyi(3000, 0.02, seed=12)
    g, og = pair(rp, col)
    k, edges = G.pattern("4-clique")
    whole = g.estimate("4-clique", scheme=api.GS, seed=31, colors=4)["exact_count"]
    cols = O.colors(og.n, 4, 31).astype(np.uint64)
    v = np.arange(og.n, dtype=np.uint64)
    total = 0
    for r in range(world):
        cnt = g.gs_count_classes("4-clique", 4, 31, r, world)
        masked = np.where(cols % world == r, cols, np.uint64(0xFFFFFFFF) - v).astype(np.uint32)
        row, cc = O.sparsify(og, masked)
        assert cnt == O.exact_count(O.Graph(row, cc), O.plan(k, edges))
        total += cnt
    assert total == whole > 0


@pytest.mark.parametrize("name,eps", [("4-clique", 0.005), ("triangle", 0.005), ("4-cycle", 0.002)])
def test_pilot_sample_count_predicts_the_online_run(name, eps):
    """The hybrid's NS cost rests on N_s = (z sd / (eps mu))^2 from a pilot
    round (Sec. 4.3 with Eq. equ:error): the online run to the same target
    needs about that many samples (within window rounding and the pilot's
    sampling error)."""
    rp, col = G.rmat(14, 16, seed=3)
    g = api.Graph(rp.cuda(), col.cuda())
    info = g.hybrid_model(name, eps=eps, delta=0.01, seed=3, window=1 << 16)
    r = g.estimate(name, eps=eps, delta=0.01, seed=3, window=1 << 14, n_max=1 << 32)
    assert r["converged"] == 1 and info["n_s"] > 8 * (1 << 14)
    assert 0.5 < r["samples"] / info["n_s"] < 2.0, (r["samples"], info["n_s"])


@pytest.mark.parametrize("name,c", [("triangle", 2), ("4-cycle", 3)])
def test_gs_sampler_variance_follows_the_corrected_model(name, c):
    """The spread of R independent GPU colourings (the sample standard deviation
    behind the R-sampler interval) against the corrected variance model of
    the oracle (pairs of matches sharing z vertices add c^(z-1) - 1)."""
    from oracle import brute, gs_variance
    rp, col = G.erdos_renyi(22, 0.4, seed=6)
    g, og = pair(rp, col)
    k, edges = G.pattern(name)
    ms = brute.matches(*G.to_numpy(rp, col), k, edges)
    var_model = float(gs_variance.colour_variance(ms, k, c))
    R, delta = 3000, 0.01
    r = g.estimate(name, scheme=api.GS, seed=9, delta=delta, colors=c, samplers=R)
    z = O.phi_inv(1 - delta / 2)
    s2 = (r["ci_half_width"] * math.sqrt(R) / z) ** 2
    assert abs(r["estimate"] - len(ms)) < 5 * math.sqrt(var_model / R)
    assert s2 == pytest.approx(var_model, rel=0.2), (s2, var_model)
