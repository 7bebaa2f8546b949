"""Pins of the Gaussian-mixture sampling prior oracle (``oracle.gmm``) and of the
three-member portfolio against what the mathematics fixes.  CPU only.

* The normal inverse CDF equals scipy's to 1e-15 (tails to 1e-300).
* The truncated mixture density integrates to 1 over the cube (the density itself on
  lines through a point of the cube and six adaptive quadratures per component, not its
  closed-form normalisation).
* Draws follow the density: component frequencies follow the weights and every
  dimension's histogram follows the mixture's marginal (closed-form bin masses).
* One weighted EM step on many draws from a mixture whose components lie well inside the
  cube returns its parameters within their sampling error (the maximum-likelihood fixed
  point); zero weight on a component keeps it.
* A GMM-only portfolio and the three-member portfolio integrate the three-Gaussian
  mixture (the paper's demonstration target) to its analytic ln Z within 4 sigma, and the
  three-member mixture density is the density of its draws (L = 1, fixed weights).
"""
import copy
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def GM(oracle_lib):
    from oracle import gmm
    return gmm


def _random_gmm(GM, C=3, seed=2):
    rng = np.random.default_rng(seed)
    g = GM.GMM(n_comp=C, seed=17)
    g.pi = rng.uniform(0.2, 1.0, C)
    g.pi /= g.pi.sum()
    g.mu = rng.uniform(0.0, 1.0, (C, 6))
    g.sig = rng.uniform(0.05, 0.6, (C, 6))
    return g


def test_ndtri_against_scipy(oracle_lib):
    from scipy.special import ndtri
    L = oracle_lib.lib()
    ps = np.concatenate([np.logspace(-300, -1, 60), np.linspace(0.01, 0.99, 99), 1 - np.logspace(-16, -1, 30)])
    for p in ps:
        x, y = L.orc_ndtri(p), ndtri(p)
        assert abs(x - y) <= 2e-15 * max(1.0, abs(y)), (p, x, y)
    assert L.orc_ndtri(0.0) == -math.inf and L.orc_ndtri(1.0) == math.inf


def test_density_integrates_to_one(GM):
    """For one component, ln g(v) is a sum of one-dimensional terms, so with v0 a point
    of the cube  int g dv = g(v0) prod_d int g(v0 with v_d = x) / g(v0) dx:  the density
    itself (as a black box, on lines through v0) and six adaptive quadratures.  A mixture
    integrates to the weighted sum of its components."""
    from scipy.integrate import quad
    g = _random_gmm(GM)
    v0 = np.full((1, 6), 0.37)
    total = 0.0
    for c in range(g.C):
        one = GM.GMM(n_comp=1)
        one.pi = np.ones(1)
        one.mu, one.sig = g.mu[c:c + 1].copy(), g.sig[c:c + 1].copy()
        l0 = one.ln_density(v0)[0]
        prod = math.exp(l0)
        for d in range(6):
            def line(x, d=d):
                v = v0.copy()
                v[0, d] = x
                return math.exp(one.ln_density(v)[0] - l0)
            val, _ = quad(line, 0.0, 1.0, epsabs=1e-13, epsrel=1e-12, limit=200)
            prod *= val
        total += g.pi[c] * prod
    assert abs(total - 1.0) < 1e-9


def _marginal_bin_masses(g, d, edges):
    from scipy.special import ndtr
    out = np.zeros(len(edges) - 1)
    for c in range(g.C):
        m, s = g.mu[c, d], g.sig[c, d]
        Z = ndtr((1 - m) / s) - ndtr(-m / s)
        out += g.pi[c] * np.diff(ndtr((edges - m) / s)) / Z
    return out


def test_draws_follow_the_density(GM):
    g = _random_gmm(GM)
    n = 200000
    th, v, comp = g.draw(n, it=3)
    assert v.min() >= 0.0 and v.max() < 1.0
    for c in range(g.C):
        f = np.mean(comp == c)
        assert abs(f - g.pi[c]) < 5 * math.sqrt(g.pi[c] * (1 - g.pi[c]) / n), (c, f, g.pi[c])
    edges = np.linspace(0, 1, 21)
    for d in range(6):
        counts = np.histogram(v[:, d], edges)[0]
        expect = n * _marginal_bin_masses(g, d, edges)
        assert np.all(np.abs(counts - expect) < 5 * np.sqrt(expect) + 1), d
    # theta is the prior mapping of v
    assert np.allclose(th[:, 0], 2 * np.pi * v[:, 0]) and np.allclose(np.sin(th[:, 1]), 2 * v[:, 1] - 1)


def test_em_fixed_point_and_dead_component(GM):
    g = GM.GMM(n_comp=2, seed=5, eps=0.0)
    g.pi = np.array([0.3, 0.7])
    g.mu = np.array([[0.3, 0.6, 0.4, 0.5, 0.35, 0.65], [0.7, 0.35, 0.6, 0.45, 0.6, 0.3]])
    g.sig = np.array([[0.04] * 6, [0.06] * 6])
    n = 400000
    _, v, comp = g.draw(n, it=0)
    h = copy.deepcopy(g)
    h.em_update(v, np.zeros(n))
    assert np.allclose(h.pi, g.pi, atol=5 * math.sqrt(0.21 / n))
    for c in range(2):
        nc = g.pi[c] * n
        assert np.all(np.abs(h.mu[c] - g.mu[c]) < 5 * g.sig[c] / math.sqrt(nc)), c
        assert np.all(np.abs(h.sig[c] - g.sig[c]) < 5 * g.sig[c] / math.sqrt(2 * nc)), c
    # a component that no weighted sample supports keeps its means and widths
    k = copy.deepcopy(g)
    k.mu[1] = 0.98
    k.sig[1] = 0.001
    lnw = np.where(comp == 0, 0.0, -np.inf)
    k.em_update(v, lnw)
    assert np.array_equal(k.mu[1], np.full(6, 0.98)) and np.array_equal(k.sig[1], np.full(6, 0.001))


def test_gmm_and_three_member_portfolios_meet_analytic_lnZ(oracle_lib):
    import sys
    import os
    sys.path.insert(0, os.path.dirname(__file__))
    import test_oracle_portfolio as T
    from oracle import portfolio as PF
    truth = T._mixture_lnZ()
    for kw in (dict(members=(False, False, True), w_init=(0, 0, 1)),
               dict(members=(True, True, True), w_init=(1 / 3, 1 / 3, 1 / 3))):
        res = PF.run(T._mixture, 12, 20000, seed=3, n_min_star=300, gmm_components=4, **kw)
        r = res["pooled"]
        assert abs(r["lnZ"] - truth) < 4 * r["sigma_lnZ"], (kw, r, truth)
        late = PF.reduce(np.concatenate([it["lnw"] for it in res["iterations"][-4:]]))
        assert abs(late["lnZ"] - truth) < 4 * late["sigma_lnZ"] and late["n_eff"] > 1000, (kw, late, truth)
        for it in res["iterations"]:
            act = np.array(kw["members"])
            assert abs(it["W"].sum() - 1) < 1e-14 and it["W"][act].min() >= 0.05 / act.sum() - 1e-15


def test_three_member_mixture_density_is_the_density_of_the_draws(oracle_lib, GM):
    """L = 1 and fixed W = (0.3, 0.3, 0.4): the weighted draws give the volume of the AV
    cells and of the rest of the cube."""
    import sys
    import os
    sys.path.insert(0, os.path.dirname(__file__))
    import test_oracle_portfolio as T
    from oracle import av as A
    from oracle import portfolio as PF
    rng = np.random.default_rng(5)
    pf = PF.Portfolio(members=(True, True, True), adapt_weights=False, w_init=(0.3, 0.3, 0.4), seed=21, n_bins=16)
    pf.hist.P = rng.uniform(0.2, 1.0, (6, 16))
    pf.hist.P /= pf.hist.P.sum(axis=1, keepdims=True)
    pf.av.level = 2
    pf.av.cells = np.unique(A.cell_keys(rng.random((40, 6)), 2))
    pf.av.V = pf.av.cells.size * 4.0 ** -6
    pf.gmm = _random_gmm(GM, C=3, seed=8)
    av_before = copy.deepcopy(pf.av)
    n = 400000
    rec = pf.step(T._flat, n)
    w = np.exp(rec["lnw"])
    inA = av_before.contains(rec["v"])
    for f, want in ((np.ones(n), 1.0), (inA, av_before.V), (~inA, 1.0 - av_before.V)):
        x = w * f
        assert abs(x.mean() - want) < 5 * x.std() / math.sqrt(n), (x.mean(), want)
    assert all(0 < k < n for k in rec["n_drawn"])
