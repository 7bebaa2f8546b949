"""Pins of the portfolio oracle (Sec. IV, "Portfolio integrator") against what the paper
and the mathematics fix.  CPU only.

* A single-member portfolio is that member: the histogram sampler and the AV integrator
  reproduced bit for bit (pins the plumbing: counters, training order, estimator).
* The mixture density is the density of the draws: with L = 1 the weighted draws
  integrate any region to its volume, inside and outside the AV member's cells, and the
  draws' marginal follows the mixture's (a wrong p_s, e.g. each member's own, biases the
  region outside the AV cells by the factor W_hist, which the test shows).
* Three-Gaussian mixture in four dimensions (the paper's demonstration target): pooled
  ln Z meets the analytic integral (erf masses in the cube).
* The weight rules: water-filling floor at 0.05/N_s, the freeze rule below 5%, the
  activation iteration.
"""
import copy
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def PF(oracle_lib):
    from oracle import portfolio
    return portfolio


def _flat(th, v):
    return np.zeros(th.shape[0])


def test_floor_weights_water_filling(PF):
    act2 = np.array([True, True])
    assert np.allclose(PF.floor_weights([0.01, 0.99], act2, 0.025), [0.025, 0.975], rtol=0, atol=1e-15)
    assert np.allclose(PF.floor_weights([3.0, 1.0], act2, 0.025), [0.75, 0.25], rtol=0, atol=1e-15)
    # scaling the rest down pushes a second weight under the floor: both end at the floor
    act3 = np.array([True, True, True])
    w = PF.floor_weights([0.05, 0.21, 0.74], act3, 0.2)
    assert np.allclose(w, [0.2, 0.2, 0.6], rtol=0, atol=1e-15)
    # inactive members get 0, the floor applies among the active ones
    w = PF.floor_weights([0.0, 5.0, 1e-9], np.array([False, True, True]), 0.05 / 2)
    assert w[0] == 0.0 and w[2] == 0.025 and abs(w.sum() - 1.0) < 1e-15


def test_member_choice_follows_the_weight(oracle_lib):
    """Draw i goes to the histogram member with probability W_hist; different
    iterations give independent choices."""
    from oracle import _p, lib
    n = 200000
    m = {}
    for g, w0 in ((0, 0.3), (1, 0.3), (2, 0.9)):
        m[g] = np.empty(n, np.int32)
        lib().orc_portfolio_members(11, g, n, w0, 2.0, _p(m[g]))
        frac = float(np.mean(m[g] == 0))
        assert abs(frac - w0) < 5 * math.sqrt(w0 * (1 - w0) / n)
    agree = float(np.mean(m[0] == m[1]))
    assert abs(agree - (0.3 ** 2 + 0.7 ** 2)) < 5 * math.sqrt(0.25 / n)
    # W = 1 and W = 0 are exact
    lib().orc_portfolio_members(11, 3, n, 1.0, 2.0, _p(m[0]))
    lib().orc_portfolio_members(11, 3, n, 0.0, 2.0, _p(m[1]))
    assert np.all(m[0] == 0) and np.all(m[1] == 1)


def _peak(th, v, sig=0.08):
    mu = np.array([0.3, 0.6, 0.45, 0.55, 0.4, 0.7])
    return -np.sum((v - mu) ** 2, 1) / (2 * sig ** 2)


def _sharp(th, v):
    return _peak(th, v, 0.02)


def test_histogram_only_portfolio_is_the_histogram_sampler(oracle_lib, PF):
    from oracle import Sampler
    pf = PF.Portfolio(members=(True, False), seed=9, n_bins=32)
    s = Sampler(n_bins=32, seed=9)
    for g in range(4):
        rec = pf.step(_peak, 20000)
        th, lr, bins, v = s.draw(20000, want_v=True)
        lnw = _peak(th, v) + lr
        s.adapt(bins, lnw)
        s.iteration += 1
        assert np.array_equal(rec["theta"], th) and np.array_equal(rec["lnw"], lnw)
        assert np.all(rec["member"] == 0) and rec["frozen"][1] and not rec["frozen"][0]
        assert np.array_equal(pf.hist.P, s.P)


def test_av_only_portfolio_is_the_av_integrator(oracle_lib, PF):
    from oracle import av as A
    pf = PF.Portfolio(members=(False, True), seed=9, n_min_star=200)
    a = A.AV(seed=9, n_min_star=200)
    for g in range(5):
        rec = pf.step(_sharp, 20000)
        th, v = a.draw(20000)
        ll = _sharp(th, v)
        lnw = ll + math.log(a.V)
        a.update(v, ll)
        assert np.array_equal(rec["theta"], th) and np.array_equal(rec["lnw"], lnw)
        assert np.all(rec["member"] == 1)
        assert (pf.av.level, pf.av.cells.size, pf.av.V) == (a.level, a.cells.size, a.V)
    assert a.level >= 2


def _shaped_portfolio(PF, W):
    """A portfolio with a non-uniform histogram (random masses) and an AV member on a
    strict subset of the level-2 grid (40 random cells), weights fixed at W."""
    rng = np.random.default_rng(5)
    pf = PF.Portfolio(adapt_weights=False, w_init=W, seed=21, n_bins=16)
    pf.hist.P = rng.uniform(0.2, 1.0, (6, 16))
    pf.hist.P /= pf.hist.P.sum(axis=1, keepdims=True)
    from oracle import av as A
    pf.av.level = 2
    pf.av.cells = np.unique(A.cell_keys(rng.random((40, 6)), 2))
    pf.av.V = pf.av.cells.size * 4.0 ** -6
    return pf


def test_mixture_density_is_the_density_of_the_draws(oracle_lib, PF):
    """L = 1 and fixed W = (0.35, 0.65): the mean weight is 1, the weighted draws give
    the volume of the AV cells and of the rest of the cube, and the draws' v_0 marginal
    is the mixture's.  Each member's own density in place of the mixture would estimate
    the region outside the AV cells at W_hist times its volume."""
    W = (0.35, 0.65)
    n = 400000
    pf = _shaped_portfolio(PF, W)
    av_before = copy.deepcopy(pf.av)
    P0 = pf.hist.P.copy()
    rec = pf.step(_flat, n)
    w = np.exp(rec["lnw"])
    inA = av_before.contains(rec["v"])
    VA = av_before.V
    for f, want in ((np.ones(n), 1.0), (inA, VA), (~inA, 1.0 - VA)):
        x = w * f
        est, err = x.mean(), x.std() / math.sqrt(n)
        assert abs(est - want) < 5 * err, (est, want, err)
    # each member's own density in place of the mixture: biased outside the AV cells
    own = np.where(rec["member"] == 0, np.exp(-pf_own_lnd(P0, rec)), av_before.V)
    x = own * ~inA
    assert abs(x.mean() - W[0] * (1 - VA)) < 5 * x.std() / math.sqrt(n)
    assert abs(x.mean() - (1 - VA)) > 20 * x.std() / math.sqrt(n)
    # the v_0 marginal: histogram bins of width 1/16, AV cells of width 1/4
    B = 16
    marg_h = P0[0] / P0[0].sum()
    c0 = (av_before.cells & np.uint64(3)).astype(int)
    marg_av = np.array([np.sum(c0 == (b * 4) // B) for b in range(B)]) / (4.0 * av_before.cells.size)
    expect = W[0] * marg_h + W[1] * marg_av
    counts = np.bincount(np.minimum((rec["v"][:, 0] * B).astype(int), B - 1), minlength=B)
    assert np.all(np.abs(counts - n * expect) < 5 * np.sqrt(n * expect))


def pf_own_lnd(P, rec):
    """ln g_hist of each draw under masses P (the test's own product of bin masses)."""
    B = P.shape[1]
    b = np.minimum((rec["v"] * B).astype(int), B - 1)
    return np.sum([np.log(B * P[d, b[:, d]] / P[d].sum()) for d in range(6)], axis=0)


# three Gaussians in the first four coordinates (flat in the other two), one broad
MU = np.array([[0.3, 0.6, 0.4, 0.7], [0.7, 0.3, 0.6, 0.3], [0.5, 0.5, 0.5, 0.5]])
SIG = np.array([0.03, 0.05, 0.2])
AMP = np.array([0.5, 0.3, 0.2])


def _mixture(th, v):
    t = [math.log(a) - np.sum((v[:, :4] - mu) ** 2, 1) / (2 * s * s) - 4 * math.log(s * math.sqrt(2 * math.pi))
         for mu, s, a in zip(MU, SIG, AMP)]
    return np.logaddexp.reduce(np.array(t), axis=0)


def _mixture_lnZ():
    def phi(x):
        return 0.5 * (1.0 + math.erf(x / math.sqrt(2.0)))
    return math.log(sum(a * np.prod([phi((1 - m) / s) - phi(-m / s) for m in mu]) for mu, s, a in zip(MU, SIG, AMP)))


def test_three_gaussian_mixture_lnZ(oracle_lib, PF):
    """The portfolio of {histogram, AV} on the three-Gaussian mixture: the pooled ln Z of
    twelve iterations of 20000 draws, and of the last four, meet the analytic value within
    4 sigma; the weights sum to 1, never fall below 0.05/2, and each batch's member counts
    follow them."""
    truth = _mixture_lnZ()
    res = PF.run(_mixture, 12, 20000, seed=3, n_min_star=300)
    r = res["pooled"]
    assert abs(r["lnZ"] - truth) < 4 * r["sigma_lnZ"], (r, truth)
    late = PF.reduce(np.concatenate([it["lnw"] for it in res["iterations"][-4:]]))
    assert abs(late["lnZ"] - truth) < 4 * late["sigma_lnZ"] and late["n_eff"] > 100, (late, truth)
    for it in res["iterations"]:
        W = it["W"][:2]   # the two active members
        assert abs(W.sum() - 1) < 1e-14 and W.min() >= 0.025 - 1e-15 and it["W"][2] == 0.0
        k = it["n_drawn"][0]
        assert abs(k - 20000 * W[0]) < 6 * math.sqrt(20000 * W[0] * W[1])
    # the weights moved away from the initial (1/2, 1/2)
    assert any(abs(it["W"][0] - 0.5) > 0.1 for it in res["iterations"][1:])


def test_freeze_rule_below_five_percent(oracle_lib, PF):
    """A member whose weight is below 0.05 is not trained: with W fixed at (0.97, 0.03)
    the AV state stays as it was while the histogram adapts; with (0.03, 0.97) the
    histogram masses stay while the AV refines."""
    pf = PF.Portfolio(adapt_weights=False, w_init=(0.97, 0.03), seed=4, n_min_star=100)
    P0 = pf.hist.P.copy()
    for _ in range(3):
        rec = pf.step(_peak, 20000)
        assert rec["frozen"].tolist() == [False, True, True] and rec["n_drawn"][1] > 0
    assert (pf.av.level, pf.av.cells.size, pf.av.V, pf.av.live_lnL.size) == (0, 1, 1.0, 0)
    assert not np.array_equal(pf.hist.P, P0)
    pf = PF.Portfolio(adapt_weights=False, w_init=(0.03, 0.97), seed=4, n_min_star=100)
    for _ in range(3):
        rec = pf.step(_peak, 20000)
        assert rec["frozen"].tolist() == [True, False, True]
    assert np.array_equal(pf.hist.P, np.full((6, 64), 1.0 / 64)) and pf.av.level >= 1


def test_av_member_joins_at_its_start_iteration(oracle_lib, PF):
    pf = PF.Portfolio(av_start=2, w_init=(0.4, 0.6), seed=6, n_min_star=100)
    for g in range(4):
        rec = pf.step(_peak, 10000)
        if g < 2:
            assert np.all(rec["member"] == 0) and rec["W"].tolist() == [1.0, 0.0, 0.0]
            assert rec["frozen"][1] and pf.av.level == 0
        elif g == 2:
            assert np.allclose(rec["W"], [0.4, 0.6, 0.0], rtol=0, atol=1e-15)
            assert 0 < rec["n_drawn"][0] < 10000
