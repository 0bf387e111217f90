"""Learned proposal on the GPU against the CPU oracle: scores and learned
samples bit-exact, FP32 training gradients within 1e-3, training rows exact,
the learned online estimate on the oracle's samples, and what the trained
network gains over plain NS (hit rate and per-sample variance) while staying
unbiased."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2405_03488_gb300 import api
from paper_2405_03488_gb300 import graphs as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2405_03488_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def oracle_weights(prop):
    return O.Weights16(*prop.arrays16())


def assert_same_records(gpu, cpu, k):
    for f in ("hit", "depth", "w_u64", "overflow"):
        bad = np.nonzero(gpu[f] != cpu[f])[0]
        assert len(bad) == 0, (f, bad[:5])
    assert np.array_equal(gpu["w_f64"].view(np.uint64), cpu["w_f64"].view(np.uint64))
    assert np.array_equal(gpu["factor"][:, :k], cpu["factor"][:, :k])
    assert np.array_equal(gpu["vert"][:, :k], cpu["vert"][:, :k])
    assert np.array_equal(gpu["aux"][:, :k], cpu["aux"][:, :k])


def test_scores_bit_exact():
    rp, col = G.complete(5)
    g = api.Graph(rp.cuda(), col.cuda())
    rng = np.random.default_rng(0)
    feat = np.concatenate([rng.uniform(0, 22, (3000, 3)),
                           np.stack([rng.integers(0, 20, 500), rng.integers(2, 9, 500),
                                     rng.integers(0, 20, 500)], 1)]).astype(np.float32)
    for seed in (1, 2, 3):
        prop = api.Proposal(seed=seed)
        got = prop.scores(g, torch.from_numpy(feat).cuda()).cpu().numpy()
        w = oracle_weights(prop)
        want = np.array([O.score(O.mlp_logit(w, list(map(float, f)))) for f in feat])
        assert np.array_equal(got.astype(np.int64), want.astype(np.int64))
        assert got.min() >= 1 and got.max() <= 4097


LEARNED = [("4-clique", False), ("5-clique", False), ("diamond", True), ("house", False), ("4-cycle", False),
           ("tailed-triangle", True), ("6-clique", False)]


@pytest.mark.parametrize("name,induced", LEARNED)
def test_learned_traces_bit_exact(name, induced):
    rp, col = G.erdos_renyi(60, 0.35, seed=8)
    g = api.Graph(rp.cuda(), col.cuda())
    og = O.Graph(*G.to_numpy(rp, col))
    prop = api.Proposal(seed=4)
    k, edges = G.pattern(name)
    gpu = g.trace((k, edges, induced), seed=21, first=777, count=2000, mlp=prop)
    _, cpu = O.ns_run(og, O.plan(k, edges, induced), seed=21, first=777, count=2000, mode=O.LEARNED,
                      mlp=oracle_weights(prop), trace=True)
    assert_same_records(gpu, cpu, k)
    assert (gpu["aux"][:, 2] > 0).any()


def test_learned_large_sets_fall_back_bit_exact():
    rp, col = G.complete(300)
    g = api.Graph(rp.cuda(), col.cuda())
    og = O.Graph(*G.to_numpy(rp, col))
    prop = api.Proposal(seed=6)
    gpu = g.trace("4-clique", seed=2, first=0, count=300, mlp=prop, cap=64)
    _, cpu = O.ns_run(og, O.plan(*G.clique(4)), seed=2, first=0, count=300, mode=O.LEARNED,
                      mlp=oracle_weights(prop), trace=True)
    assert_same_records(gpu, cpu, 4)
    sizes, learned = gpu["factor"][:, 2], gpu["aux"][:, 2] > 0
    assert learned.any() and ((~learned) & (sizes > 256)).any()


def test_loss_and_gradient_match_oracle():
    rp, col = G.complete(5)
    g = api.Graph(rp.cuda(), col.cuda())
    rng = np.random.default_rng(3)
    for rows in (1, 63, 64, 1000, 5000):
        feat = rng.uniform(0, 12, (rows, 3)).astype(np.float32)
        label = (rng.uniform(size=rows) < 0.4).astype(np.float32)
        prop = api.Proposal(seed=rows)
        loss, grad = prop.loss_grad(g, torch.from_numpy(feat).cuda(), torch.from_numpy(label).cuda())
        w = prop.w32.cpu().numpy()
        w32 = {"w1": w[0:192].reshape(64, 3), "b1": w[192:256], "w2": w[256:4352].reshape(64, 64),
               "b2": w[4352:4416], "w3": w[4416:4480], "b3": w[4480:4481]}
        oloss, og_ = O.mlp_loss_grad(w32, feat, label)
        assert loss == pytest.approx(oloss, rel=1e-3)
        flat = np.concatenate([og_[k].ravel() for k in ("w1", "b1", "w2", "b2", "w3", "b3")])
        gg = grad.cpu().numpy()
        scale = np.abs(flat).max()
        assert np.max(np.abs(gg - flat)) <= 1e-3 * scale + 1e-7


def test_training_rows_from_traces_exact():
    rp, col = G.erdos_renyi(80, 0.3, seed=2)
    g = api.Graph(rp.cuda(), col.cuda())
    og = O.Graph(*G.to_numpy(rp, col))
    deg = np.diff(G.to_numpy(rp, col)[0])
    for name in ("5-clique", "house"):
        k, edges = G.pattern(name)
        recs = g.trace(name, seed=3, first=0, count=4000)
        dev = torch.from_numpy(recs.view(np.uint8).copy()).cuda()
        feat, label = api.proposal_features(g, name, dev, len(recs))
        want_f, want_l = [], []
        for r in recs:
            for j in range(2, k - 1):
                if r["hit"] or r["depth"] > j:
                    want_f.append([O.flog2p1(int(deg[r["vert"][j]])), float(j), O.flog2p1(int(r["factor"][j + 1]))])
                    reached = k if r["hit"] else int(r["depth"])
                    want_l.append(np.float32(reached - j - 1) / np.float32(k - j - 1))
        assert np.array_equal(feat.cpu().numpy(), np.array(want_f, dtype=np.float32).reshape(-1, 3))
        assert np.array_equal(label.cpu().numpy(), np.array(want_l, dtype=np.float32))


def test_learned_online_matches_oracle():
    # untrained weights make the importance weights extreme, so the run stops
    # at n_max; the rounds, totals and predicted error still match the oracle
    rp, col = G.erdos_renyi(400, 0.1, seed=5)
    g = api.Graph(rp.cuda(), col.cuda())
    og = O.Graph(*G.to_numpy(rp, col))
    prop = api.Proposal(seed=9)
    W = 1 << 13
    r = g.estimate("5-clique", scheme=api.NS_LEARNED, eps=0.05, delta=0.01, seed=4, window=W, n_max=6 * W,
                   mlp=prop)
    o = O.ns_online(og, O.plan(*G.clique(5)), 0.05, 0.01, seed=4, window=W, n_max=6 * W, mode=O.LEARNED,
                    mlp=oracle_weights(prop))
    assert r["scheme_used"] == api.NS_LEARNED
    assert r["converged"] == o.converged == 0
    assert (r["samples"], r["hits"], r["rounds"]) == (o.samples, o.hits, o.rounds) == (6 * W, o.hits, 6)
    assert r["estimate"] == pytest.approx(o.estimate, rel=1e-12)
    assert r["eps_hat"] == pytest.approx(o.eps_hat, rel=1e-10)


def test_trained_proposal_gains_over_plain_and_stays_unbiased():
    """Train on plain-NS traces of a power-law graph with planted cliques, then
    compare per-sample variance and hit rate with plain NS on fresh seeds."""
    rp, col = G.chung_lu(200_000, n_cliques=200, clique_size=12, seed=4, device="cuda")
    g = api.Graph(rp, col)
    name = "6-clique"
    exact = g.exact_count(name)
    prop = api.Proposal(seed=1)
    loss, rows = prop.train(g, name, seed=11, samples=1 << 20, epochs=3, batch=8192, lr=3e-3)
    assert rows > 1000 and np.isfinite(loss)
    N = 1 << 22
    plain = g.sample_sums(name, seed=101, first=0, count=N)
    learned = g.sample_sums(name, seed=101, first=0, count=N, mlp=prop)

    def stats(s):
        mu = s.sum / s.n
        return mu, max(s.sumsq / s.n - mu * mu, 0.0), s.hits / s.n

    mp, vp, hp = stats(plain)
    ml, vl, hl = stats(learned)
    # unbiased: both within 5 standard errors of the exact count
    assert abs(mp - exact) < 5 * math.sqrt(vp / N) + 1e-9 * exact
    assert abs(ml - exact) < 5 * math.sqrt(vl / N) + 1e-9 * exact
    # the gain: more hits and a smaller per-sample variance
    assert hl > hp
    assert vl < vp


# ------------------------------------------------------------------ tensor-core scoring (mlp_tensor = 1)
def _bf16_round(x):
    """Round float32 values to BF16 (nearest even), returned as float64."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def test_tensor_core_scores_within_the_bf16_bound():
    """The tensor-core scores differ from the FP32 oracle's only through the BF16
    rounding of the layer-1 outputs (relative error <= 2^-9 each) and the
    summation order: per row, |dz| <= sum_o |w3_o| (2^-8 sum_i |W2_oi h1_i|) +
    2^-18 sum_o |w3_o h2_o|, and a = 1 + floor(512 z + 2048) moves by at most
    512 |dz| + 1."""
    rp, col = G.complete(5)
    g = api.Graph(rp.cuda(), col.cuda())
    rng = np.random.default_rng(4)
    feat = np.concatenate([rng.uniform(0, 22, (2000, 3)),
                           np.stack([rng.integers(0, 20, 500), rng.integers(2, 9, 500),
                                     rng.integers(0, 20, 500)], 1)]).astype(np.float32)
    for seed in (1, 2):
        prop = api.Proposal(seed=seed)
        got = prop.scores(g, torch.from_numpy(feat).cuda(), tensor=True).cpu().numpy().astype(np.int64)
        w = oracle_weights(prop)
        want = np.array([O.score(O.mlp_logit(w, list(map(float, f)))) for f in feat], dtype=np.int64)
        w16 = [np.asarray(a, dtype=np.uint16) for a in prop.arrays16()]
        f32 = [(a.astype(np.uint32) << 16).view(np.float32).astype(np.float64) for a in w16]
        w1, b1, w2, b2, w3 = f32[0].reshape(64, 3), f32[1], f32[2].reshape(64, 64), f32[3], f32[4]
        h1 = np.maximum(feat.astype(np.float64) @ w1.T + b1, 0.0)
        h2 = np.maximum(h1 @ w2.T + b2, 0.0)
        dz = (np.abs(h1) @ np.abs(w2).T) @ np.abs(w3) * 2.0 ** -8 + (np.abs(h2) @ np.abs(w3)) * 2.0 ** -18
        bound = np.floor(512 * dz) + 1
        diff = np.abs(got - want)
        assert np.all(diff <= bound), (diff.max(), bound[diff.argmax()])
        assert got.min() >= 1 and got.max() <= 4097
        # the tensor path reads the BF16-rounded hidden layer: its exact logits are closer still
        zr = (np.maximum(_bf16_round(h1) @ w2.T + b2, 0.0) @ w3 + f32[5][0])
        ar = 1 + np.floor(4096 * np.clip(zr / 8 + 0.5, 0, 1))
        assert np.all(np.abs(got - ar) <= 1 + np.floor(512 * (np.abs(h2) @ np.abs(w3)) * 2.0 ** -18) + 1)


def test_tensor_core_learned_sampler_is_unbiased():
    """Any positive scores keep the estimator unbiased: the tensor-core learned
    sampler's mean over 2^20 samples lies within 5 standard errors of the
    exact count, and each sample's weight is A / a_x times the uniform steps."""
    rp, col = G.erdos_renyi(300, 0.12, seed=6)
    g = api.Graph(rp.cuda(), col.cuda())
    og = O.Graph(*G.to_numpy(rp, col))
    for name in ("4-clique", "house"):
        k, edges = G.pattern(name)
        exact = O.exact_count(og, O.plan(k, edges))
        prop = api.Proposal(seed=3)
        N = 1 << 20
        s = g.sample_sums(name, seed=7, first=0, count=N, mlp=prop, mlp_tensor=1)
        mu = s.sum / s.n
        var = max(s.sumsq / s.n - mu * mu, 0.0)
        assert abs(mu - exact) < 5 * math.sqrt(var / N), (name, mu, exact)
        tr = g.trace(name, seed=7, first=0, count=4096, mlp=prop, mlp_tensor=1)
        hit = tr["hit"] == 1
        w = tr["factor"][:, 0].astype(np.float64)
        for j in range(2, k):
            learned = tr["aux"][:, j] > 0
            fj = tr["factor"][:, j].astype(np.float64)
            w = w * np.where(learned, fj / np.maximum(tr["aux"][:, j], 1), fj)
        assert np.allclose(tr["w_f64"][hit], w[hit], rtol=1e-12)
        assert hit.sum() > 0 and (tr["aux"][hit, 2] > 0).any()


def test_one_adam_step_matches_the_host_step():
    """One training step on one full batch is Adam's first step written out on
    the host: m = 0.1 g, v = 0.001 g^2, w -= lr (m / 0.1) / (sqrt(v / 0.001) + 1e-8),
    with g the mean-loss gradient at the starting weights (gpm_mlp_loss_grad)."""
    rp, col = G.complete(5)
    g = api.Graph(rp.cuda(), col.cuda())
    rng = np.random.default_rng(8)
    feat = torch.from_numpy(rng.uniform(0, 12, (500, 3)).astype(np.float32)).cuda()
    label = torch.from_numpy((rng.random(500) < 0.3).astype(np.float32)).cuda()
    prop = api.Proposal(seed=6)
    w0 = prop.w32.clone()
    _, grad = prop.loss_grad(g, feat, label)
    lr = 1e-2
    prop.train_rows(g, feat, label, epochs=1, batch=500, lr=lr)
    gg = grad.double().cpu().numpy()
    m, v = 0.1 * gg, 0.001 * gg * gg
    want = w0.double().cpu().numpy() - lr * (m / 0.1) / (np.sqrt(v / 0.001) + 1e-8)
    got = prop.w32.double().cpu().numpy()
    assert np.allclose(got, want, rtol=2e-6, atol=1e-9)
    # the BF16 copies are the FP32 weights rounded to nearest even
    bits = prop.w32.cpu().numpy().view(np.uint32).astype(np.uint64)
    rne = ((bits + 0x7FFF + ((bits >> 16) & 1)) >> 16).astype(np.uint16)
    assert np.array_equal(prop.w16.cpu().numpy().view(np.uint16), rne)


def test_bf16_copies_keep_nan():
    """A NaN weight (here the output bias) spreads NaN to every weight whose
    gradient it reaches; the BF16 copies of those must be NaN too, not
    infinities or zeros, and every finite weight keeps its nearest-even copy."""
    rp, col = G.complete(5)
    g = api.Graph(rp.cuda(), col.cuda())
    feat = torch.ones((64, 3), dtype=torch.float32, device="cuda")
    label = torch.zeros(64, dtype=torch.float32, device="cuda")
    prop = api.Proposal(seed=6)
    prop.w32[4480] = float("nan")
    prop.train_rows(g, feat, label, epochs=1, batch=64, lr=1e-2)
    w32 = prop.w32.cpu().numpy()
    w16 = prop.w16.cpu().numpy().view(np.uint16).astype(np.uint32)
    nan = np.isnan(w32)
    assert nan.sum() > 64
    assert np.all((w16[nan] & 0x7F80) == 0x7F80) and np.all((w16[nan] & 0x7F) != 0)
    bits = w32[~nan].view(np.uint32).astype(np.uint64)
    assert np.array_equal(w16[~nan], ((bits + 0x7FFF + ((bits >> 16) & 1)) >> 16).astype(np.uint32))
