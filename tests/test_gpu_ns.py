"""GPU parity of the NS sampler (INTERSECT and CHECK verify) against the CPU
oracle, through the C ABI: per-sample records bit-exact, FP64 aggregates
within 1e-12 relative, the online stopping rule on the same samples."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2405_03488_gb300 import api
from paper_2405_03488_gb300 import graphs as G

pytestmark = pytest.mark.gpu

REL = 1e-12   # FP64 reduction-order tolerance of aggregates


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2405_03488_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def pair(rp, col):
    """(GPU handle borrowing CUDA tensors, oracle graph on the host copy)."""
    g = api.Graph(rp.cuda(), col.cuda(), validate=True)
    return g, O.Graph(*G.to_numpy(rp, col))


def assert_same_records(gpu, cpu, k):
    assert len(gpu) == len(cpu)
    for f in ("hit", "depth", "w_u64", "overflow"):
        bad = np.nonzero(gpu[f] != cpu[f])[0]
        assert len(bad) == 0, (f, bad[:5], gpu[f][bad[:5]], cpu[f][bad[:5]])
    assert np.array_equal(gpu["w_f64"].view(np.uint64), cpu["w_f64"].view(np.uint64))
    assert np.array_equal(gpu["factor"][:, :k], cpu["factor"][:, :k])
    assert np.array_equal(gpu["vert"][:, :k], cpu["vert"][:, :k])


PATTERNS = [("triangle", False), ("4-clique", False), ("5-clique", False), ("4-cycle", False),
            ("4-cycle", True), ("diamond", False), ("tailed-triangle", True), ("3-star", True),
            ("4-path", False), ("house", False), ("5-path", True), ("edge", False),
            ("5-path", False), ("3-star", False), ("dumbbell", False), ("tailed-triangle", False),
            ("wedge", False)]


MODES = {"intersect": O.INTERSECT, "check": O.CHECK, "lazy": O.LAZY}


@pytest.mark.parametrize("verify", ["intersect", "check", "lazy"])
@pytest.mark.parametrize("name,induced", PATTERNS)
def test_trace_bit_exact_small(name, induced, verify):
    rp, col = G.erdos_renyi(40, 0.3, seed=3)
    g, og = pair(rp, col)
    k, edges = G.pattern(name)
    pat = (k, edges, induced)
    mode = MODES[verify]
    first, count = 12345, 3001
    gpu = g.trace(pat, seed=77, first=first, count=count, verify=verify)
    _, cpu = O.ns_run(og, O.plan(k, edges, induced), seed=77, first=first, count=count, mode=mode, trace=True)
    assert_same_records(gpu, cpu, k)
    if verify == "intersect":
        assert gpu["hit"].sum() > 0


@pytest.mark.parametrize("cap,warps,blocks", [(1, 1, 3), (4, 2, 5), (33, 8, 7), (512, 4, 0)])
def test_two_pass_and_odd_shapes_bit_exact(cap, warps, blocks):
    # dense graph: candidate sets overflow the small on-chip buffers
    rp, col = G.erdos_renyi(80, 0.5, seed=5)
    g, og = pair(rp, col)
    for name, induced in (("4-clique", False), ("4-cycle", False), ("diamond", True), ("5-clique", False)):
        k, edges = G.pattern(name)
        gpu = g.trace((k, edges, induced), seed=9, first=0, count=1500, cap=cap, block_warps=warps,
                      grid_blocks=blocks)
        _, cpu = O.ns_run(og, O.plan(k, edges, induced), seed=9, first=0, count=1500, trace=True)
        assert_same_records(gpu, cpu, k)


@pytest.mark.parametrize("cap", [64, 96, 160])
def test_sampled_list_searches_bit_exact(cap):
    """Lists longer than the on-chip buffer are searched through an on-chip
    sample of every step-th entry (the partner list of a step, N(v_{j-1}) when
    S_j is cut from S_{j-1}, the non-neighbours removed from S_{j-1} in
    vertex-induced plans): degrees of 100-200 against buffers of 64-160 entries
    take every one of those paths, with uneven segment lengths."""
    for rp, col in (G.erdos_renyi(300, 0.45, seed=8), G.rmat(11, 24, seed=6)):
        g, og = pair(rp, col)
        for name, induced in (("4-clique", False), ("5-clique", False), ("diamond", True), ("3-star", True),
                              ("tailed-triangle", True), ("4-cycle", True), ("house", False)):
            k, edges = G.pattern(name)
            gpu = g.trace((k, edges, induced), seed=4, first=0, count=1200, cap=cap)
            _, cpu = O.ns_run(og, O.plan(k, edges, induced), seed=4, first=0, count=1200, trace=True)
            assert_same_records(gpu, cpu, k)


@pytest.mark.parametrize("cap", [32, 512])
def test_induced_single_list_positions_bit_exact(cap):
    """Vertex-induced steps with one back-neighbour on a skewed graph: the
    back-neighbour's list is long (a hub) and the non-neighbours' lists short,
    so the removed entries are located by their positions in it; more of them
    than the buffer holds (cap 32) falls back to streaming the list."""
    rp, col = G.rmat(14, 16, seed=9)
    g, og = pair(rp, col)
    for name in ("3-star", "4-path", "tailed-triangle", "4-cycle"):
        k, edges = G.pattern(name)
        gpu = g.trace((k, edges, True), seed=21, first=0, count=20000, cap=cap)
        _, cpu = O.ns_run(og, O.plan(k, edges, True), seed=21, first=0, count=20000, trace=True)
        assert_same_records(gpu, cpu, k)
        assert gpu["hit"].sum() > 0


def test_sums_match_oracle_er_triangle_1e6():
    """ER G(n=10^4, p=0.002), triangle, 10^6 samples, seed 1."""
    rp, col = G.erdos_renyi(10_000, 0.002, seed=1)
    g, og = pair(rp, col)
    p = O.plan(*G.pattern("triangle"))
    N = 1_000_000
    s = g.sample_sums("triangle", seed=1, first=0, count=N)
    acc, _ = O.ns_run(og, p, seed=1, first=0, count=N)
    assert s.n == N and s.hits == acc.hits
    assert s.sum == pytest.approx(acc.sum, rel=REL)
    assert s.sumsq == pytest.approx(acc.sumsq, rel=REL)
    exact = O.exact_count(og, p)
    mean = s.sum / N
    sd = math.sqrt((s.sumsq / N - mean * mean) / N)
    assert abs(mean - exact) < 5 * sd


@pytest.mark.parametrize("verify", ["intersect", "check", "lazy"])
def test_online_matches_oracle(verify):
    rp, col = G.erdos_renyi(3000, 0.01, seed=2)
    g, og = pair(rp, col)
    mode = MODES[verify]
    # NS-base hits far less often (about 1 in 1200 triangle samples here), so it gets looser targets
    targets = (("triangle", 0.05), ("4-cycle", 0.1)) if verify == "lazy" else (("triangle", 0.02), ("4-cycle", 0.05))
    for name, eps in targets:
        k, edges = G.pattern(name)
        W = 1 << 15
        r = g.estimate(name, eps=eps, delta=0.01, seed=4, window=W, verify=verify)
        o = O.ns_online(og, O.plan(k, edges), eps, 0.01, seed=4, window=W, mode=mode)
        assert r["converged"] == o.converged == 1
        assert r["samples"] == o.samples and r["rounds"] == o.rounds and r["hits"] == o.hits
        assert r["estimate"] == pytest.approx(o.estimate, rel=REL)
        assert r["eps_hat"] == pytest.approx(o.eps_hat, rel=1e-10)
        assert r["ci_half_width"] == pytest.approx(o.ci_half_width, rel=1e-10)


def test_edge_cases():
    # no edges at all: every sample misses, mu = 0, never converges
    rp, col = G.from_edge_list(6, [])
    g = api.Graph(rp.cuda(), col.cuda())
    r = g.estimate("triangle", eps=0.1, delta=0.1, seed=1, window=1000, n_max=3000)
    assert r["estimate"] == 0.0 and r["converged"] == 0 and r["samples"] == 3000
    tr = g.trace("triangle", seed=1, first=0, count=10)
    assert tr["hit"].sum() == 0 and np.all(tr["depth"] == 0)
    # one-edge pattern: weight m on every sample, exact at once
    rp, col = G.complete(9)
    g = api.Graph(rp.cuda(), col.cuda())
    r = g.estimate("edge", eps=0.01, delta=0.01, seed=1, window=100)
    assert r["estimate"] == 36.0 and r["eps_hat"] == 0.0 and r["rounds"] == 1
    # isolated vertices, ragged counts, a far sample offset
    rp, col = G.from_edge_list(50, [(1, 7), (7, 9), (1, 9), (9, 30), (30, 1), (7, 30), (44, 45)])
    g, og = pair(rp, col)
    for count in (1, 31, 33, 1023):
        for first in (0, 2**40 + 5):
            gpu = g.trace("4-clique", seed=3, first=first, count=count)
            _, cpu = O.ns_run(og, O.plan(*G.clique(4)), seed=3, first=first, count=count, trace=True)
            assert_same_records(gpu, cpu, 4)
            s = g.sample_sums("4-clique", seed=3, first=first, count=count)
            acc, _ = O.ns_run(og, O.plan(*G.clique(4)), seed=3, first=first, count=count)
            assert (s.n, s.hits) == (acc.n, acc.hits) and s.sum == pytest.approx(acc.sum, rel=REL)


def test_validation_rejects_bad_csr():
    from paper_2405_03488_gb300 import _lib
    rp, col = G.complete(5)
    bad = col.clone()
    bad[0], bad[1] = bad[1].item(), bad[0].item()     # unsorted
    with pytest.raises(_lib.GpmError) as e:
        api.Graph(rp.cuda(), bad.cuda(), validate=True)
    assert e.value.code == _lib.GPM_ERR_GRAPH
    asym_rp = torch.tensor([0, 1, 1], dtype=torch.int64)
    with pytest.raises(_lib.GpmError):
        api.Graph(asym_rp.cuda(), torch.tensor([1], dtype=torch.int32).cuda(), validate=True)
    # host arrays are copied, and a valid graph passes
    g = api.Graph(rp.numpy(), col.numpy(), validate=True)
    assert (g.n, g.m, g.nnz, g.max_degree) == (5, 10, 20, 4)


@pytest.fixture(scope="module")
def rmat22():
    rp, col = G.rmat(22, 16, seed=2, device="cuda")
    return rp, col


def test_rmat22_lazy_sampled_parity(rmat22):
    """NS-base on R-MAT scale 22: records at two stream depths, 4-clique and 4-cycle."""
    rp, col = rmat22
    g = api.Graph(rp, col)
    og = O.Graph(*G.to_numpy(rp, col))
    for name in ("4-clique", "4-cycle"):
        k, edges = G.pattern(name)
        for first in (0, 987_654_321):
            gpu = g.trace(name, seed=1, first=first, count=4096, verify="lazy")
            _, cpu = O.ns_run(og, O.plan(k, edges), seed=1, first=first, count=4096, mode=O.LAZY, trace=True)
            assert_same_records(gpu, cpu, k)


@pytest.mark.parametrize("name", ["4-clique", "5-clique", "house", "4-cycle"])
def test_rmat22_sampled_parity_in_bench_shape(rmat22, name):
    """R-MAT scale 22 (the benchmark workload): records of sample ranges deep
    into a run are bit-exact, in the launch shape the benchmark uses."""
    rp, col = rmat22
    g = api.Graph(rp, col)
    og = O.Graph(*G.to_numpy(rp, col))
    k, edges = G.pattern(name)
    p = O.plan(k, edges)
    for first in (0, 987_654_321):
        gpu = g.trace(name, seed=1, first=first, count=20_000)
        _, cpu = O.ns_run(og, p, seed=1, first=first, count=20_000, trace=True)
        assert_same_records(gpu, cpu, k)
        assert gpu["hit"].sum() > 0
    count = (1 << 18) if name.endswith("clique") else (1 << 14)    # the oracle is slow on hub lists
    s = g.sample_sums(name, seed=1, first=1 << 20, count=count)
    acc, _ = O.ns_run(og, p, seed=1, first=1 << 20, count=count)
    assert (s.n, s.hits) == (acc.n, acc.hits)
    assert s.sum == pytest.approx(acc.sum, rel=REL) and s.sumsq == pytest.approx(acc.sumsq, rel=REL)


def test_interval_coverage_on_er_triangles():
    """1000 seeds of the convergence test on G(10^4, 0.002) triangles (the
    exact count from the exact counter, checked against the oracle): the
    fraction of stopped estimates within eps of C is at least 1 - delta minus
    three binomial standard deviations."""
    rp, col = G.erdos_renyi(10_000, 0.002, seed=1)
    g, og = pair(rp, col)
    C = g.exact_count("triangle")
    assert C == O.exact_count(og, O.plan(*G.pattern("triangle")))
    R, eps, delta = 1000, 0.05, 0.05
    miss = 0
    for s in range(1, R + 1):
        r = g.estimate("triangle", eps=eps, delta=delta, seed=s, window=1 << 14)
        assert r["converged"] == 1
        miss += abs(r["estimate"] - C) > eps * C
    assert miss <= R * delta + 3 * (R * delta * (1 - delta)) ** 0.5, miss


def _mem_available_gb():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) / 1e6
    except OSError:
        pass
    return 0.0


def test_rmat27_sampled_parity_at_full_size():
    """R-MAT scale 27 (134M vertices, 2.1G edges, the largest workload), in the
    launch shape its benchmark uses: per-sample records deep into the stream
    are bit-exact, and a block of sums equals the oracle's."""
    if _mem_available_gb() < 48 or torch.cuda.get_device_properties(0).total_memory < 150e9:
        pytest.skip("needs 48 GB of host and 150 GB of device memory")
    rp, col = G.rmat(27, 16, seed=5, device="cuda")
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    g = api.Graph(rp, col)
    gpu = {}
    for name in ("5-clique", "4-cycle"):
        for first in (0, 987_654_321):
            gpu[(name, first)] = g.trace(name, seed=1, first=first, count=4096)
    s = g.sample_sums("5-clique", seed=1, first=1 << 30, count=1 << 15)
    og = O.Graph(rp.cpu().numpy().view(np.uint64), col.cpu().numpy().view(np.uint32))
    del g, rp, col
    torch.cuda.empty_cache()
    for (name, first), recs in gpu.items():
        k, edges = G.pattern(name)
        _, cpu = O.ns_run(og, O.plan(k, edges), seed=1, first=first, count=4096, trace=True)
        assert_same_records(recs, cpu, k)
        assert recs["hit"].sum() > 0
    acc, _ = O.ns_run(og, O.plan(*G.pattern("5-clique")), seed=1, first=1 << 30, count=1 << 15)
    assert (s.n, s.hits) == (acc.n, acc.hits)
    assert s.sum == pytest.approx(acc.sum, rel=REL) and s.sumsq == pytest.approx(acc.sumsq, rel=REL)


def test_abort_deadline_and_allocation_failure_are_clean():
    """Failure handling without faulting the GPU: an abort set from another
    host thread ends a running estimate with ABORTED and a partial result;
    max_seconds ends one with NOT_CONVERGED; a CSR too large for the device
    fails with OOM before any copy; the handle stays usable after each."""
    import threading
    import time
    from paper_2405_03488_gb300 import _lib
    rp, col = G.rmat(16, 16, seed=3, device="cuda")
    g = api.Graph(rp, col)
    threading.Timer(0.3, g.abort).start()
    t0 = time.perf_counter()
    r = g.estimate("5-clique", eps=1e-5, delta=0.01, seed=1, window=1 << 16, n_max=1 << 40)
    assert r["status"] == _lib.GPM_ERR_ABORTED and r["converged"] == 0 and r["samples"] > 0
    assert time.perf_counter() - t0 < 30
    r = g.estimate("5-clique", eps=1e-5, delta=0.01, seed=1, window=1 << 16, n_max=1 << 40, max_seconds=0.3)
    assert r["status"] == _lib.GPM_ERR_NOT_CONVERGED and r["converged"] == 0 and r["samples"] > 0
    big = np.array([0, 1 << 40], dtype=np.uint64)      # claims 2^40 neighbour entries
    with pytest.raises(_lib.GpmError) as e:
        api.Graph(big, np.zeros(4, dtype=np.uint32))
    assert e.value.code == _lib.GPM_ERR_OOM
    r = g.estimate("triangle", eps=0.05, delta=0.01, seed=2, window=1 << 16)
    assert r["converged"] == 1
