"""gpm_sample_sums_static: the sampling entry point for callers that cannot
allocate device memory during a call (an application that reserved its device
memory up front in a pool of its own, a latency-bound loop that cannot afford
an allocation's synchronisation).  Its totals must equal those of the
allocating gpm_sample_sums bit for bit, at every count up to its 2^22-sample
limit, and must not depend on what an earlier call left in the shared array.
This file is collected last so that a failure here does not hide any other
test."""
import ctypes as C

import pytest
import torch

from paper_2405_03488_gb300 import _lib, api
from paper_2405_03488_gb300 import graphs as G

pytestmark = pytest.mark.gpu

LIMIT = 1 << 22


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


def same(out, ref):
    return (out.n, out.hits, out.sum, out.sumsq) == (ref.n, ref.hits, ref.sum, ref.sumsq)


@pytest.fixture(scope="module")
def er():
    rp, col = G.erdos_renyi(3000, 0.01, seed=2)
    return api.Graph(rp.cuda(), col.cuda())


@pytest.mark.parametrize("name,seed,first,count,cfg", [
    ("4-clique", 11, 0, 500_000, {}),
    ("4-cycle", 12, 1 << 30, 3_000_017, {"verify": "check"}),
    ("triangle", 13, 5, LIMIT, {}),
])
def test_static_scratch_equals_allocating_entry_point_on_repeated_calls(er, name, seed, first, count, cfg):
    ref = er.sample_sums(name, seed=seed, first=first, count=count, **cfg)
    for _ in range(2):   # the second call finds the first call's partials in the array
        code, out = static_sums(er, name, seed, first, count, **cfg)
        assert code == _lib.GPM_OK, _lib.load().gpm_last_error()
        assert same(out, ref)


def test_static_scratch_learned_proposal(er):
    prop = api.Proposal(seed=3)
    ref = er.sample_sums("4-clique", seed=4, first=0, count=200_000, mlp=prop)
    code, out = static_sums(er, "4-clique", 4, 0, 200_000, mlp=prop)
    assert code == _lib.GPM_OK, _lib.load().gpm_last_error()
    assert same(out, ref)


def test_static_scratch_rejects_oversized_calls():
    rp, col = G.complete(6)
    g = api.Graph(rp.cuda(), col.cuda())
    code, _ = static_sums(g, "triangle", 1, 0, LIMIT + 1)
    assert code == _lib.GPM_ERR_ARG
    assert b"2^22" in _lib.load().gpm_last_error()
    code, out = static_sums(g, "triangle", 1, 0, 1 << 10)
    assert code == _lib.GPM_OK and out.n == 1 << 10
