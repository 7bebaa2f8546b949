"""Adaptive-volume integrator (rift_ile_av) against the oracle's step-by-step AV.

With the float64 path every discrete decision (draw cell, live set, threshold bin,
grid level, active cells) is taken on values that agree with the oracle's to ~1e-12,
so the state after every iteration is compared exactly, the draws to the last-bit
differences of the inverse-CDF transcendentals, and ln Z to 1e-9 relative.
"""
import math

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


@pytest.mark.parametrize("problem", ["plain", "large"])
def test_av_fp64_matches_oracle_step_by_step(G, orc, problem):
    from oracle import av as A
    p = S.plain_fp64_problem() if problem == "plain" else S.single_large_problem()
    n, iters = 20000, 5
    kw = dict(p_thr=0.999, n_min_star=300)
    a = A.AV(seed=13, capacity=4 * n, d_min=p.d_min, d_max=p.d_max, **kw)
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=n, seed=13) as s:
        for g in range(iters):
            r = s.av(1, n, capacity=4 * n, restart=(g == 0), **kw)
            info = s.av_info()
            th, lr, ll, lw = s.last_batch(n)
            rec = a.step(lambda t: orc.lnL(p, t), n)
            assert np.allclose(th, rec["theta"], rtol=1e-12, atol=1e-14), g
            assert np.all(lr == math.log(rec["V"]))
            assert np.max(np.abs(ll - rec["lnL"]) / np.maximum(1, np.abs(rec["lnL"]))) < 1e-9
            assert (info["level"], info["n_cells"], info["n_live"], info["V"]) == \
                (a.level, a.cells.size, a.live_lnL.size, a.V), (g, info)
            red = orc.reduce(rec["lnw"])
            assert abs(r["lnZ"] - red["lnZ"]) <= 1e-9 * max(1.0, abs(red["lnZ"]))
    assert a.level >= 2   # the grid refined


def test_av_fp32_refines_and_meets_oracle(G, orc):
    """Five AV iterations in float32 on the single large problem: the active volume
    shrinks from one iteration to the next once the grid refines, and the last
    iteration's ln Z on the device's own draws is within 1e-3 of the oracle's float64
    reduction."""
    p = S.single_large_problem()
    n = 30000
    vols = []
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=n, seed=17) as s:
        for g in range(5):
            r = s.av(1, n, p_thr=0.999, n_min_star=500, restart=(g == 0))
            vols.append(s.av_info()["V"])
        info = s.av_info()
        th, lr, ll, lw = s.last_batch(n)
    assert info["level"] >= 2 and vols[-1] < 0.05
    assert all(b <= a for a, b in zip(vols, vols[1:]))
    red = orc.reduce(orc.lnL(p, th) + lr)
    assert abs(r["lnZ"] - red["lnZ"]) <= 1e-3


def high_snr_realisable(G, snr=150.0, point=0):
    """SNR-150 injection with the q=20-like hierarchy (3 detectors, 21 modes, 16384 Hz,
    1001 bins), built from the library's float64 coefficients at a near-edge-on truth so
    that the injection is realisable."""
    th_true = np.array([2.2, -0.5, 1.1, 0.7, 1.4, 300.0])
    probe = S.high_snr_problem(snr=snr, point=point)
    with G.ILE(probe, precision=G.RIFT_FP64, max_samples=16) as s:
        c, dt, _ = s.coeffs(th_true[None, :])
    return S.high_snr_problem(snr=snr, point=point, a0=c[0] * th_true[5] / probe.d_ref, dt_true=dt[0])


@pytest.mark.slow
def test_av_high_snr_agrees_with_histogram_sampler(G, orc):
    """The high-SNR workload (SNR 150, sharply peaked likelihood), RIFT_MIXED: ten AV
    iterations of 1e6 draws against the histogram sampler's late iterations (its
    iterations 20..29 of 1e6 samples, combined by inverse variance).  With N_min* a floor
    the AV live set does not collapse onto the first iteration's few best draws: the last
    AV iteration's ln Z is within 4 combined sigma + 1e-3 of the histogram sampler's, and
    on its own draws within 1e-3 of the float64 oracle's reduction."""
    p = high_snr_realisable(G)
    n = 1_000_000
    with G.ILE(p, precision=G.RIFT_MIXED, max_samples=n, n_bins=64, seed=1) as s:
        rh = s.adapt(30, n)
    zh, sh = np.array(rh["lnZ_iter"][20:]), np.array(rh["sigma_iter"][20:])
    wgt = 1.0 / sh ** 2
    z_hist, s_hist = float(np.sum(wgt * zh) / np.sum(wgt)), float(1.0 / np.sqrt(np.sum(wgt)))
    with G.ILE(p, precision=G.RIFT_MIXED, max_samples=n, n_bins=64, seed=1) as s:
        ra = s.av(10, n, p_thr=0.9999, n_min_star=1000, restart=True)
        th, lr, ll, lw = s.last_batch(n)
    z_av, s_av = ra["lnZ_iter"][-1], ra["sigma_iter"][-1]
    assert ra["n_eff_iter"][-1] > 20
    assert abs(z_av - z_hist) <= 4.0 * math.hypot(s_av, s_hist) + 1e-3, (z_av, s_av, z_hist, s_hist)
    # parity of the last AV iteration on its own draws: RIFT_MIXED re-evaluates in float64
    # every draw within 40 of the largest ln w (all the weight): those against the oracle to
    # 1e-3, and ln Z with the oracle's values in their place
    heavy = np.nonzero(lw >= lw.max() - 40.0)[0]
    oll = orc.lnL(p, th[heavy])
    assert np.max(np.abs(ll[heavy] - oll)) <= 1e-3
    lnw = ll + lr
    lnw[heavy] = oll + lr[heavy]
    red = orc.reduce(lnw)
    assert abs(z_av - red["lnZ"]) <= 1e-3


def test_av_arguments_and_state(G):
    p = S.plain_fp64_problem()
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=1000, seed=1) as s:
        for bad in (dict(n_per_iter=2000), dict(p_thr=0.0), dict(p_thr=1.5), dict(n_min_star=0),
                    dict(capacity=10)):
            kw = dict(n_iter=1, n_per_iter=1000, p_thr=0.99, n_min_star=10, capacity=4000, restart=1)
            kw.update(bad)
            with pytest.raises(G.RiftError) as e:
                G.rift_ile_av(s.h, kw["n_iter"], kw["n_per_iter"], kw["p_thr"], kw["n_min_star"], kw["capacity"],
                              kw["restart"])
            assert e.value.code == G.RIFT_EINVAL
        s.av(2, 1000, capacity=4000)
        with pytest.raises(G.RiftError) as e:
            s.av(1, 1000, capacity=8000)   # capacity is fixed by the first call
        assert e.value.code == G.RIFT_EINVAL
        before = s.av_info()
        s.av(1, 1000, capacity=4000, restart=True)
        assert s.av_info()["level"] <= before["level"] or before["level"] == 0
        # fair draws work on the AV batch
        th, t, idx = s.fair_draws(100, seed=2)
        assert th.shape == (100, 6)
