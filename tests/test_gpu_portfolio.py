"""Portfolio integrator (rift_ile_portfolio) against the oracle's step-by-step portfolio,
over {histogram, AV} and over {histogram, AV, Gaussian mixture}.

With the float64 path every discrete decision (member choice, histogram bin, AV cell,
live set, threshold, grid level, weight floor, freeze) is taken on values that agree with
the oracle's to ~1e-10, so the state after every iteration is compared exactly, the draws
to the last-bit differences of the inverse-CDF transcendentals, the weights, n_ESS and
ln Z to 1e-9 relative in the first iteration.  Once the histogram masses are trained
(they agree to ~1e-10) the histogram draws agree to 1e-6 and the weights to 1e-4, while
the AV member's state stays exact, and every ln L and ln Z on the device's own draws meet
the oracle to 1e-9.  The float32 path is held to the float32 bar (1e-3) on its own
draws.  Single-member portfolios reproduce the library's own samplers exactly.  The
Gaussian mixture's draws use the device's normal quantile against the oracle's Newton
iteration on the same probability (a few ulps apart), and its parameters after each EM
step meet the oracle's to the rounding of sums taken in another order.
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


def _rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.maximum(1.0, np.abs(np.asarray(b)))))


@pytest.mark.parametrize("problem,av_start", [("plain", 0), ("large", 0), ("large", 2)])
def test_portfolio_fp64_matches_oracle_step_by_step(G, orc, problem, av_start):
    from oracle import portfolio as PF
    p = S.plain_fp64_problem() if problem == "plain" else S.single_large_problem()
    n, iters, B = 20000, 6, 32
    kw = dict(p_thr=0.999, n_min_star=300)
    pf = PF.Portfolio(seed=13, n_bins=B, capacity=4 * n, av_start=av_start, w_init=(0.5, 0.5), d_min=p.d_min,
                      d_max=p.d_max, **kw)
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=n, n_bins=B, seed=13) as s:
        for g in range(iters):
            r = s.portfolio(1, n, capacity=4 * n, av_start=av_start, restart=(g == 0), **kw)
            info = s.portfolio_info()
            av = s.av_info()
            th, lr, ll, lw = s.last_batch(n)
            rec = pf.step(lambda t, v: orc.lnL(p, t), n)
            assert info["iteration"] == g + 1
            if g < av_start:
                assert info["n_drawn"] == [n, 0, 0] and info["active"] == [1, 0, 0]
            assert info["n_drawn"] == rec["n_drawn"].tolist(), g
            # before any training the two draw streams agree to the last bits; afterwards the
            # histogram masses agree to ~1e-10 (weighted sums of a wide dynamic range in
            # another order), which moves a histogram draw in a light bin by up to ~1e-7
            first = g == 0
            assert np.allclose(th, rec["theta"], rtol=1e-12 if first else 1e-6, atol=1e-12 if first else 1e-9), g
            assert _rel(lr, rec["lr"]) < (1e-11 if first else 1e-6), g
            assert np.allclose(info["W_last"], rec["W"], rtol=1e-12 if first else 1e-6, atol=1e-15), (g, info)
            assert np.allclose(info["W_next"], rec["W_next"], rtol=1e-9 if first else 1e-4, atol=1e-12), (g, info)
            assert np.allclose(info["n_ess"], rec["n_ess"], rtol=1e-9 if first else 1e-4, atol=1e-9), (g, info)
            assert info["frozen"] == rec["frozen"].astype(int).tolist(), g
            # the AV member learns from its own draws, which do not depend on the masses: exact
            assert (av["level"], av["n_cells"], av["n_live"], av["V"]) == \
                (pf.av.level, pf.av.cells.size, pf.av.live_lnL.size, pf.av.V), (g, av)
            red = orc.reduce(rec["lnw"])
            assert abs(r["lnZ"] - red["lnZ"]) <= (1e-9 if first else 1e-4) * max(1.0, abs(red["lnZ"])), g
            # on the device's own draws: every ln L and the reduction to 1e-9
            oll = orc.lnL(p, th)
            assert _rel(ll, oll) < 1e-9, g
            own = orc.reduce(oll + lr)
            assert abs(r["lnZ"] - own["lnZ"]) <= 1e-9 * max(1.0, abs(own["lnZ"])), g
            assert abs(r["n_ess"] - own["n_ess"]) <= 1e-9 * own["n_ess"], g
    assert pf.av.level >= 1


def test_portfolio_fp32_meets_oracle_on_its_draws(G, orc):
    """Five float32 iterations on the single large problem: the weights stay normalised
    and above 0.05/2, both members draw, and the last iteration's ln Z on the device's own
    draws is within 1e-3 of the oracle's float64 reduction of those draws."""
    p = S.single_large_problem()
    n = 30000
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=n, seed=17) as s:
        for g in range(5):
            r = s.portfolio(1, n, p_thr=0.999, n_min_star=500, restart=(g == 0))
            info = s.portfolio_info()
            assert abs(sum(info["W_next"]) - 1.0) < 1e-12 and min(info["W_next"][:2]) >= 0.025 - 1e-15
            assert min(info["n_drawn"][:2]) > 0 and sum(info["n_drawn"]) == n and info["W_next"][2] == 0.0
        th, lr, ll, lw = s.last_batch(n)
    oll = orc.lnL(p, th)
    assert np.max(np.abs(ll - oll)) <= 1e-3
    red = orc.reduce(oll + lr)
    assert abs(r["lnZ"] - red["lnZ"]) <= 1e-3


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_single_member_portfolios_are_the_library_samplers(G, precision):
    """Histogram alone reproduces rift_ile_adapt, AV alone rift_ile_av, iteration by
    iteration (the same draws, weights and training)."""
    p = S.single_large_problem()
    prec = G.RIFT_FP64 if precision == "fp64" else G.RIFT_FP32
    n, iters = 20000, 4
    with G.ILE(p, precision=prec, max_samples=n, n_bins=32, seed=5) as s:
        ra = s.adapt(iters, n)
    with G.ILE(p, precision=prec, max_samples=n, n_bins=32, seed=5) as s:
        rp = s.portfolio(iters, n, members=G.RIFT_MEMBER_HIST, restart=True)
        info = s.portfolio_info()
    assert rp["lnZ_iter"] == ra["lnZ_iter"] and rp["lnZ"] == ra["lnZ"]
    assert info["n_drawn"] == [n, 0, 0] and info["frozen"] == [0, 1, 1]
    with G.ILE(p, precision=prec, max_samples=n, seed=5) as s:
        rv = s.av(iters, n, p_thr=0.999, n_min_star=300, capacity=4 * n, restart=True)
        av1 = s.av_info()
    with G.ILE(p, precision=prec, max_samples=n, seed=5) as s:
        rq = s.portfolio(iters, n, members=G.RIFT_MEMBER_AV, p_thr=0.999, n_min_star=300, capacity=4 * n,
                         restart=True)
        av2 = s.av_info()
    assert rq["lnZ_iter"] == rv["lnZ_iter"] and av1 == av2


def test_portfolio_arguments(G):
    p = S.plain_fp64_problem()
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=1000, seed=1) as s:
        bad = [dict(members=0), dict(members=8), dict(members=G.RIFT_MEMBER_AV, av_start=1), dict(av_start=-1),
               dict(members=G.RIFT_MEMBER_GMM, gmm_start=1), dict(members=7, gmm_start=-1),
               dict(members=G.RIFT_MEMBER_AV | G.RIFT_MEMBER_GMM, av_start=2, gmm_start=1),
               dict(members=7, gmm_components=0), dict(members=7, gmm_components=G.RIFT_GMM_MAX_COMPONENTS + 1),
               dict(w_init=(0.0, 1.0)), dict(w_init=(1.0, float("nan"))), dict(members=7, w_init=(1.0, 1.0, 0.0)),
               dict(p_thr=0.0), dict(n_min_star=0), dict(capacity=10), dict(n_per_iter=2000)]
        for b in bad:
            kw = dict(n_iter=1, n_per_iter=1000, capacity=4000)
            kw.update(b)
            with pytest.raises(G.RiftError) as e:
                s.portfolio(**kw)
            assert e.value.code == G.RIFT_EINVAL, b
        s.portfolio(2, 1000, capacity=4000, restart=True)
        with pytest.raises(G.RiftError) as e:
            s.portfolio(1, 1000, capacity=8000)   # the AV capacity is fixed by the first call
        assert e.value.code == G.RIFT_EINVAL
        th, t, idx = s.fair_draws(100, seed=2)   # fair draws work on the portfolio's batch
        assert th.shape == (100, 6)
        for change in (dict(members=7), dict(members=G.RIFT_MEMBER_HIST)):   # members change: restart needed
            with pytest.raises(G.RiftError) as e:
                s.portfolio(1, 1000, capacity=4000, **change)
            assert e.value.code == G.RIFT_EINVAL, change
        s.portfolio(1, 1000, capacity=4000, members=7, gmm_components=3, restart=True)
        with pytest.raises(G.RiftError) as e:
            s.portfolio(1, 1000, capacity=4000, members=7, gmm_components=5)
        assert e.value.code == G.RIFT_EINVAL
        assert s.portfolio_gmm()[1].shape == (3, 6)
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=1000, seed=1) as s:
        s.portfolio(1, 1000, capacity=4000, restart=True)
        with pytest.raises(G.RiftError) as e:
            s.portfolio_gmm()   # no GMM member yet
        assert e.value.code == G.RIFT_ESTATE
        s.portfolio(1, 1000, capacity=4000, members=7, restart=True)
        assert s.portfolio_gmm()[0].shape == (4,)
        s.portfolio(1, 1000, capacity=4000, restart=True)   # restarted without the mixture
        with pytest.raises(G.RiftError) as e:
            s.portfolio_gmm()
        assert e.value.code == G.RIFT_ESTATE
    pd = S.plain_fp64_problem()
    with G.ILE(pd, precision=G.RIFT_FP64, max_samples=1000, seed=1, distance_marg=True) as s:
        with pytest.raises(G.RiftError) as e:
            s.portfolio(1, 1000, capacity=4000)
        assert e.value.code == G.RIFT_EINVAL


@pytest.mark.parametrize("n", [1, 7, 129, 4097])
def test_portfolio_ragged_batches_match_oracle(G, orc, n):
    """Batch sizes that leave partial blocks, warps and EM tiles everywhere (including a
    single draw): three float64 iterations of the three-member portfolio follow the
    oracle's (draws, weights, member counts, ln Z, the mixture's parameters)."""
    from oracle import portfolio as PF
    p = S.plain_fp64_problem()
    kw = dict(p_thr=0.99, n_min_star=min(n, 50))
    pf = PF.Portfolio(members=(True, True, True), w_init=(1, 1, 1), gmm_components=3, seed=23, n_bins=16,
                      capacity=8 * n, d_min=p.d_min, d_max=p.d_max, **kw)
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=n, n_bins=16, seed=23) as s:
        for g in range(3):
            r = s.portfolio(1, n, members=7, gmm_components=3, capacity=8 * n, restart=(g == 0), **kw)
            info = s.portfolio_info()
            th, lr, ll, lw = s.last_batch(n)
            rec = pf.step(lambda t, v: orc.lnL(p, t), n)
            assert info["n_drawn"] == rec["n_drawn"].tolist(), (n, g)
            first = g == 0
            assert np.allclose(th, rec["theta"], rtol=1e-12 if first else 1e-6, atol=1e-12 if first else 1e-9), (n, g)
            assert np.allclose(info["W_next"], rec["W_next"], rtol=1e-9 if first else 1e-4, atol=1e-12), (n, g)
            own = orc.reduce(orc.lnL(p, th) + lr)
            assert abs(r["lnZ"] - own["lnZ"]) <= 1e-9 * max(1.0, abs(own["lnZ"])), (n, g)
            _check_gmm(s.portfolio_gmm(), rec["gmm"], 1e-9 if first else 1e-6, (n, g))


def _check_gmm(dev, ref, rtol, what):
    for name, a, b in zip(("pi", "mu", "sig"), dev, ref):
        assert a.shape == b.shape and np.allclose(a, b, rtol=rtol, atol=rtol * 1e-3), (what, name, a, b)


@pytest.mark.parametrize("problem,av_start,gmm_start", [("plain", 0, 0), ("large", 0, 0), ("large", 1, 2)])
def test_three_member_portfolio_fp64_matches_oracle_step_by_step(G, orc, problem, av_start, gmm_start):
    """Histogram, AV and Gaussian mixture (4 components) for six float64 iterations,
    the members joining at once or one after another.  A width at its 1e-3 floor makes
    the iteration map amplify rounding by ~10 per step (a state that agrees to 1e-13 after
    one step agrees to 1e-5 after six), so before every step the oracle takes the device's
    trained state (histogram masses, mixture parameters, weights; the AV state agrees
    exactly by itself) and each step is held to the first step's bar: member counts, the
    state each member decides (frozen, active, AV level and cells), the draws, weights,
    n_ESS, ln Z, and the mixture's parameters after its EM step."""
    from oracle import portfolio as PF
    p = S.plain_fp64_problem() if problem == "plain" else S.single_large_problem()
    n, iters, B, Cg = 20000, 6, 32, 4
    kw = dict(p_thr=0.999, n_min_star=300)
    w0 = (0.4, 0.3, 0.3)
    pf = PF.Portfolio(members=(True, True, True), seed=13, n_bins=B, capacity=4 * n, av_start=av_start,
                      gmm_start=gmm_start, w_init=w0, gmm_components=Cg, d_min=p.d_min, d_max=p.d_max, **kw)
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=n, n_bins=B, seed=13) as s:
        for g in range(iters):
            r = s.portfolio(1, n, members=7, capacity=4 * n, av_start=av_start, gmm_start=gmm_start,
                            gmm_components=Cg, w_init=w0, restart=(g == 0), **kw)
            info = s.portfolio_info()
            av = s.av_info()
            gm = s.portfolio_gmm()
            th, lr, ll, lw = s.last_batch(n)
            rec = pf.step(lambda t, v: orc.lnL(p, t), n)
            assert info["active"] == pf.active(g).astype(int).tolist(), g
            assert info["n_drawn"] == rec["n_drawn"].tolist(), g
            assert info["frozen"] == rec["frozen"].astype(int).tolist(), g
            # the draws to the last bits (the mixture's within a few ulps of its normal quantile)
            assert np.allclose(th, rec["theta"], rtol=1e-12, atol=1e-12), g
            assert _rel(lr, rec["lr"]) < 1e-11, g
            assert np.allclose(info["W_last"], rec["W"], rtol=1e-12, atol=1e-15), (g, info)
            assert np.allclose(info["W_next"], rec["W_next"], rtol=1e-9, atol=1e-12), (g, info)
            assert np.allclose(info["n_ess"], rec["n_ess"], rtol=1e-9, atol=1e-9), (g, info)
            assert (av["level"], av["n_cells"], av["n_live"], av["V"]) == \
                (pf.av.level, pf.av.cells.size, pf.av.live_lnL.size, pf.av.V), (g, av)
            if g < gmm_start:   # not started: the initial state, bit for bit
                assert all(np.array_equal(a, b) for a, b in zip(gm, rec["gmm"])), g
            else:
                # a width near its floor takes sum r v^2 / S - mu^2 with ~1e5 cancellation
                _check_gmm(gm, rec["gmm"], 1e-8, g)
            red = orc.reduce(rec["lnw"])
            assert abs(r["lnZ"] - red["lnZ"]) <= 1e-9 * max(1.0, abs(red["lnZ"])), g
            oll = orc.lnL(p, th)
            assert _rel(ll, oll) < 1e-9, g
            own = orc.reduce(oll + lr)
            assert abs(r["lnZ"] - own["lnZ"]) <= 1e-9 * max(1.0, abs(own["lnZ"])), g
            assert abs(r["n_ess"] - own["n_ess"]) <= 1e-9 * own["n_ess"], g
            # the next step starts from the device's trained state
            pf.hist.P = np.asarray(s.sampler(), np.float64).reshape(6, B).copy()
            pf.gmm.pi, pf.gmm.mu, pf.gmm.sig = (np.array(x) for x in gm)
            pf.W = np.array(info["W_next"])
    assert info["n_drawn"][2] > 0


@pytest.mark.parametrize("Cg", [6, 16])
def test_gmm_only_portfolio_matches_oracle(G, orc, Cg):
    """The Gaussian mixture alone (6 components, and the largest count, 16): every draw is
    its own, ln p - ln p_s is minus its log density, and it trains on every sample; four
    float64 iterations against the oracle's GMM-only portfolio."""
    from oracle import portfolio as PF
    p = S.single_large_problem()
    n = 20000
    pf = PF.Portfolio(members=(False, False, True), w_init=(0, 0, 1), gmm_components=Cg, seed=29, d_min=p.d_min,
                      d_max=p.d_max)
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=n, seed=29) as s:
        for g in range(4):
            r = s.portfolio(1, n, members=G.RIFT_MEMBER_GMM, gmm_components=Cg, restart=(g == 0))
            info = s.portfolio_info()
            th, lr, ll, lw = s.last_batch(n)
            rec = pf.step(lambda t, v: orc.lnL(p, t), n)
            first = g == 0
            assert info["n_drawn"] == [0, 0, n] and info["active"] == [0, 0, 1], g
            assert info["W_last"] == [0.0, 0.0, 1.0], g
            assert np.allclose(th, rec["theta"], rtol=1e-12 if first else 1e-6, atol=1e-12 if first else 1e-9), g
            assert _rel(lr, rec["lr"]) < (1e-11 if first else 1e-6), g
            _check_gmm(s.portfolio_gmm(), rec["gmm"], 1e-9 if first else 1e-6, g)
            own = orc.reduce(orc.lnL(p, th) + lr)
            assert abs(r["lnZ"] - own["lnZ"]) <= 1e-9 * max(1.0, abs(own["lnZ"])), g


@pytest.mark.parametrize("Cg", [4, 16])
def test_three_member_portfolio_fp32_meets_oracle_on_its_draws(G, orc, Cg):
    """Five float32 iterations of the three-member portfolio on the single large problem
    (4 and 16 mixture components): weights normalised and above 0.05/3, every member draws,
    the mixture's parameters stay in range, and the last iteration's ln L and ln Z on the
    device's own draws are within 1e-3 of the oracle's float64 values."""
    p = S.single_large_problem()
    n = 30000
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=n, seed=17) as s:
        for g in range(5):
            r = s.portfolio(1, n, members=7, gmm_components=Cg, p_thr=0.999, n_min_star=500, restart=(g == 0))
            info = s.portfolio_info()
            assert abs(sum(info["W_next"]) - 1.0) < 1e-12 and min(info["W_next"]) >= 0.05 / 3 - 1e-15
            assert min(info["n_drawn"]) > 0 and sum(info["n_drawn"]) == n
        pi, mu, sig = s.portfolio_gmm()
        th, lr, ll, lw = s.last_batch(n)
    assert abs(pi.sum() - 1.0) < 1e-12 and mu.min() >= 0.0 and mu.max() <= 1.0
    assert sig.min() >= 1e-3 and sig.max() <= 1.0
    oll = orc.lnL(p, th)
    assert np.max(np.abs(ll - oll)) <= 1e-3
    red = orc.reduce(oll + lr)
    assert abs(r["lnZ"] - red["lnZ"]) <= 1e-3
