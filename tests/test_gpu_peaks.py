"""rift_ile_peak_rate: the measured unit rates the bench's roofline fractions are taken
against are positive, finite and of the part's order of magnitude, and an unknown unit is
refused."""
import math

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2505_11655_gb300 as G
    G.load(build_if_missing=True)
    return G


def test_measured_unit_rates(G):
    # (unit, lowest and highest plausible rate on a GB300 in tera-operations per second)
    bounds = {G.RIFT_PEAK_FP32_FMA: (20.0, 200.0), G.RIFT_PEAK_TC_F16_N128: (300.0, 5000.0),
              G.RIFT_PEAK_TC_F16_N256: (300.0, 5000.0), G.RIFT_PEAK_EX2: (1.0, 100.0),
              G.RIFT_PEAK_FP64_FMA: (0.1, 100.0)}
    for what, (lo, hi) in bounds.items():
        r = G.rift_ile_peak_rate(what)
        assert math.isfinite(r) and lo <= r <= hi, (what, r)


def test_unknown_unit_refused(G):
    for what in (-1, 5):
        with pytest.raises(G.RiftError) as e:
            G.rift_ile_peak_rate(what)
        assert e.value.code == G.RIFT_EINVAL
