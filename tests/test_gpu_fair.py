"""Fair draws (rift_ile_fair_draws) against the oracle.

The oracle runs its own chain on the same seeds: its sampler's draws (the same stream
the device draws, checked elsewhere), its float64 ln L and ln w, then its fair draws.
With the float64 path the weights agree to ~1e-12, so the drawn samples' indices, their
time bins and times are compared exactly (theta to the last-bit differences of the
inverse-CDF transcendentals).  With float32 ln w the sample weights differ by
float32 rounding (~1e-4 relative on weighted samples), which moves a running-sum
boundary past a threshold in well under 1% of draws; the time bins use float64 ln L on
both sides and are compared exactly wherever the sample agrees.
"""
import numpy as np
import pytest

import ile_synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2505_11655_gb300 as G
    G.load(build_if_missing=True)
    return G


@pytest.fixture(scope="module")
def orc(oracle_lib):
    return oracle_lib


def oracle_chain(orc, p, n, sampler_seed, n_draws, draw_seed, n_bins=32):
    sm = orc.Sampler(n_bins=n_bins, seed=sampler_seed)
    th, lr, _ = sm.draw(n, it=0)
    lnw = orc.lnL(p, th) + lr
    return orc.fair_draws(p, th, lnw, n_draws, draw_seed)


@pytest.mark.parametrize("problem", ["plain", "large"])
def test_fair_draws_fp64_exact(G, orc, problem):
    p = S.plain_fp64_problem() if problem == "plain" else S.single_large_problem()
    n, n_draws = 6000, 3000
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=n, n_bins=32, seed=41) as s:
        s.marginalize(n)
        th, t, idx = s.fair_draws(n_draws, seed=99)
    oidx, oth, oj, ot = oracle_chain(orc, p, n, 41, n_draws, 99)
    assert np.array_equal(idx, oidx)
    assert np.allclose(th, oth, rtol=1e-12, atol=1e-14)   # inverse-CDF transcendentals differ in the last bit
    assert np.allclose(t, ot, rtol=0, atol=1e-15)
    # the draws follow the weights: the heaviest samples are drawn repeatedly
    assert len(np.unique(idx)) < n_draws


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_fair_draws_reduced_precision(G, orc, precision):
    prec = G.RIFT_FP32 if precision == "fp32" else G.RIFT_MIXED
    p = S.single_large_problem()
    n, n_draws = 20000, 4000
    with G.ILE(p, precision=prec, max_samples=n, n_bins=32, seed=43) as s:
        s.marginalize(n)
        th, t, idx = s.fair_draws(n_draws, seed=7)
    oidx, oth, oj, ot = oracle_chain(orc, p, n, 43, n_draws, 7)
    same = idx == oidx
    assert same.mean() >= 0.99, same.mean()
    assert np.allclose(th[same], oth[same], rtol=1e-12, atol=1e-14)
    assert np.allclose(t[same], ot[same], rtol=0, atol=1e-15)


def test_fair_draws_after_adaptation_and_edges(G, orc):
    """Draws come from the most recent batch (after 2 adaptive iterations); no batch
    yet is a state error; zero draws is a no-op; outputs may go to device memory."""
    import torch
    p = S.plain_fp64_problem()
    n = 5000
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=n, n_bins=16, seed=5) as s:
        with pytest.raises(G.RiftError) as e:
            s.fair_draws(10)
        assert e.value.code == G.RIFT_ESTATE
        s.adapt(2, n)
        bth, blr, bll, blw = s.last_batch(n)
        th, t, idx = s.fair_draws(2000, seed=3)
        G.rift_ile_fair_draws(s.h, 0, 3)
        tt = torch.empty(2000, dtype=torch.float64, device="cuda")
        ii = torch.empty(2000, dtype=torch.int64, device="cuda")
        G.rift_ile_fair_draws(s.h, 2000, 3, t=tt, index=ii)
    assert np.array_equal(ii.cpu().numpy(), idx) and np.array_equal(tt.cpu().numpy(), t)
    assert np.array_equal(th, bth[idx])
    # the oracle's own adaptive chain: its last batch agrees with the device's to the
    # float64 rounding of the adapted masses, and so do the draws
    sm = orc.Sampler(n_bins=16, seed=5)
    res = orc.run_adapt(p, sm, 2, n)
    oth_b, olnw = res["theta"][-1], res["lnw"][-1]
    assert np.allclose(bth, oth_b, rtol=1e-9, atol=1e-12)
    oidx, oth, oj, ot = orc.fair_draws(p, oth_b, olnw, 2000, 3)
    assert np.array_equal(idx, oidx) and np.allclose(t, ot, rtol=0, atol=1e-15)
