"""The random-sector gather probe behind the benchmark's second roofline:
it runs, reports a rate within physical limits, and an L2-resident buffer is
faster than one far above L2."""
import pytest
import torch

from paper_2405_03488_gb300 import api

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2405_03488_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def test_gather_probe_reports_a_plausible_rate():
    l2 = api.gather_probe(1 << 20, chain=4, hops=1 << 24)
    hbm = api.gather_probe(1 << 30, chain=4, hops=1 << 24)
    assert 1e9 < hbm < 2e13 and 1e9 < l2 < 1e14
    assert l2 > hbm


def test_gather_probe_rejects_bad_arguments():
    with pytest.raises(Exception):
        api.gather_probe(100, chain=4)
    with pytest.raises(Exception):
        api.gather_probe(1 << 20, chain=0)
