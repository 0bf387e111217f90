"""libgpm.so builds for sm_103a, loads, and exports every entry point that
include/gpm.h declares; its host-only logic (planner, normal quantile,
argument checks) is checked without a GPU."""
import os
import re

import pytest

from oracle import oracle as O
from paper_2405_03488_gb300 import _lib, api, build
from paper_2405_03488_gb300 import graphs as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(gpm_[a-z_0-9]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    L = _lib.load()
    names = declared_symbols()
    assert len(names) >= 14
    for name in names:
        assert hasattr(L, name), name
    bound = {n for n, _, _ in _lib.SIGNATURES}
    assert names <= bound, names - bound


@pytest.mark.parametrize("name", ["triangle", "wedge", "3-star", "4-path", "tailed-triangle", "4-cycle",
                                  "diamond", "4-clique", "5-clique", "5-path", "house", "dumbbell",
                                  "6-clique", "7-clique", "8-clique", "9-clique"])
def test_library_plan_matches_oracle_plan(name):
    k, edges = G.pattern(name)
    order, res, ori = api.plan(name)
    op = O.plan(k, edges)
    assert order == list(op.order[:k])
    assert sorted(res) == sorted(op.restrictions())
    assert ori == op.oriented


def test_normal_quantile_matches_scipy():
    from scipy.special import ndtri
    import numpy as np
    for p in np.concatenate([np.logspace(-300, -1, 100), np.linspace(0.01, 0.99, 99), 1 - np.logspace(-15, -2, 30)]):
        assert abs(api.normal_quantile(float(p)) - ndtri(p)) <= 2e-15 * max(1.0, abs(ndtri(p)))


def test_plan_rejects_bad_patterns():
    with pytest.raises(_lib.GpmError):
        api.plan((4, [(0, 1), (2, 3)]))          # disconnected
    with pytest.raises(_lib.GpmError):
        api.plan((11, [(i, i + 1) for i in range(10)]))   # too large
    with pytest.raises(_lib.GpmError):
        api.plan((1, []))


def test_null_arguments_are_rejected_without_a_device():
    import ctypes as C
    L = _lib.load()
    res = _lib.Result()
    assert L.gpm_estimate(None, None, 0, 0.1, 0.1, 1, None, C.byref(res)) == _lib.GPM_ERR_ARG
    assert L.gpm_load_csr(3, None, None, 0, None, None) == _lib.GPM_ERR_ARG
    assert L.gpm_abort(None) == _lib.GPM_ERR_ARG
    assert b"null" in L.gpm_last_error()
