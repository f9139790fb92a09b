"""The measurement probes behind the cold-path and repair rooflines return
plausible ceilings on the current device."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    import torch
    assert torch.cuda.is_available()
    from paper_2412_15122_gb300 import apsp, build
    build.build()
    return apsp


def test_addmin_probe(A):
    r32 = A.apsp_probe_addmin_rate(A.APSP_I32)
    rf = A.apsp_probe_addmin_rate(A.APSP_F32)
    # at least one step per SM and clock, at most the lanes of every SM per clock
    assert 1e11 < r32 < 1e15 and 1e11 < rf < 1e15


def test_l2_probe(A):
    gbs = A.apsp_probe_l2_read_gbs()
    assert 500.0 < gbs < 200000.0
