"""gpm_sample_sums_static: the sampling entry point for callers that cannot
allocate device memory during a call (stream capture, a pre-reserved memory
pool, latency-bound loops).  It must give the same totals as the allocating
gpm_sample_sums.  This file is collected last so that a failure here does not
hide any other test."""
import ctypes as C

import pytest
import torch

from paper_2405_03488_gb300 import _lib, api
from paper_2405_03488_gb300 import graphs as G

pytestmark = pytest.mark.gpu

REL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2405_03488_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def static_sums(g, name, seed, first, count, **cfg):
    L = _lib.load()
    out = _lib.Sums()
    pp = api.pattern(name)
    c = api.config(**cfg)
    code = L.gpm_sample_sums_static(g.h, C.byref(pp), seed, first, count, C.byref(c), C.byref(out))
    return code, out


def test_static_scratch_matches_allocating_entry_point_twice():
    rp, col = G.erdos_renyi(3000, 0.01, seed=2)
    g = api.Graph(rp.cuda(), col.cuda())
    calls = [("4-clique", 11, 0, 500_000, {}), ("4-cycle", 12, 1 << 30, 3_000_017, {"verify": "check"})]
    for name, seed, first, count, cfg in calls:
        ref = g.sample_sums(name, seed=seed, first=first, count=count, **cfg)
        code, out = static_sums(g, name, seed, first, count, **cfg)
        assert code == _lib.GPM_OK, _lib.load().gpm_last_error()
        assert (out.n, out.hits) == (ref.n, ref.hits)
        assert out.sum == pytest.approx(ref.sum, rel=REL)
        assert out.sumsq == pytest.approx(ref.sumsq, rel=REL)


def test_static_scratch_rejects_oversized_calls():
    rp, col = G.complete(6)
    g = api.Graph(rp.cuda(), col.cuda())
    code, _ = static_sums(g, "triangle", 1, 0, (1 << 26) + 1)
    assert code == _lib.GPM_ERR_ARG
    assert b"2^26" in _lib.load().gpm_last_error()
    code, out = static_sums(g, "triangle", 1, 0, 1 << 10)
    assert code == _lib.GPM_OK and out.n == 1 << 10
