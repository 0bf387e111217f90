"""The two sample-count profilers (gpm_profile): the pilot on G and the
paper's fast profiler on a 10%-edge-sparsified G' (Sec. 5.3), against the
samples the online run (Algorithm 3) actually takes.  Neither changes an
estimate; they feed the NS cost model."""
import math

import pytest
import torch

from paper_2405_03488_gb300 import api
from paper_2405_03488_gb300 import graphs as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2405_03488_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


@pytest.mark.parametrize("gen,name", [("er", "triangle"), ("rmat", "4-clique"), ("rmat", "4-cycle")])
def test_profilers_predict_the_online_sample_count(gen, name):
    rp, col = G.erdos_renyi(5000, 0.01, seed=2) if gen == "er" else G.rmat(15, 16, seed=2)
    g = api.Graph(rp.cuda(), col.cuda())
    eps = 0.02
    r = g.estimate(name, eps=eps, delta=0.01, seed=1, window=1 << 12, n_max=1 << 30)
    assert r["converged"] == 1
    pil = g.profile(name, kind="pilot", eps=eps, delta=0.01, seed=2, window=1 << 18)
    spa = g.profile(name, kind="sparsified", frac=0.1, eps=eps, delta=0.01, seed=2)
    for info in (pil, spa):
        assert math.isfinite(info["n_s"]) and info["n_s"] > 0 and info["seconds"] > 0
    # the pilot sees G itself: within a factor of 2
    assert 0.5 < pil["n_s"] / r["samples"] < 2.0
    # the sparsified profiler transfers the variance through the hit-rate ratio: within a factor of 10
    assert 0.1 < spa["n_s"] / r["samples"] < 10.0, (spa, r["samples"])
    assert 0 < spa["rho_g"] <= 1 and 0 < spa["rho_gp"] <= 1 and spa["eps_o"] <= 0.5
