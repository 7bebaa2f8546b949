"""Full-size runs in the launch configurations the bench times, against the oracle.

Each run's last batch of 1e6 samples is checked sample by sample where the oracle can
afford it: every sample whose ln w lies within 40 of the batch's largest (they carry all of
ln Z but a fraction below N e^-40) plus 300 at random, each to the float32 bar (1e-3 in
ln L) at SNR 20; at SNR 150 the mixed mode's bar is on the weighted samples (float64 on the
device, 1e-6 here), and the float32 values of the others are reported.  ln Z is then
rebuilt with the oracle's ln L on the heavy samples and the device's on the rest, and
compared with the device's ln Z of that iteration to 1e-3.
"""
import math

import numpy as np
import pytest

import ile_synth as S

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


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


def lse(x):
    m = np.max(x)
    return m + math.log(np.sum(np.exp(x - m)))


def check_last_batch(orc, p, th, lr, ll, lw, lnZ_dev, all_bar=1e-3, max_heavy=400000):
    """The heavy samples and 300 others against the oracle (every one to all_bar, or only
    reported when all_bar is None); ln Z rebuilt with the oracle's values of the heavy ones.
    Returns (heavy indices, oracle ln L of them, max error of the others)."""
    n = th.shape[0]
    heavy = np.nonzero(lw >= lw.max() - 40.0)[0]
    assert 0 < heavy.size <= max_heavy, heavy.size
    rest = np.setdiff1d(np.random.default_rng(11).choice(n, 300, replace=False), heavy)
    exp_h = orc.lnL(p, th[heavy])
    exp_r = orc.lnL(p, th[rest])
    d_h = np.abs(ll[heavy] - exp_h)
    d_r = np.abs(ll[rest] - exp_r)
    assert np.max(d_h) <= 1e-3, (float(np.max(d_h)), int(heavy[np.argmax(d_h)]))
    if all_bar is not None and rest.size:
        assert np.max(d_r) <= all_bar, (float(np.max(d_r)), int(rest[np.argmax(d_r)]))
    lnw = ll + lr
    lnw[heavy] = exp_h + lr[heavy]
    lnZ = lse(lnw) - math.log(n)
    assert abs(lnZ - lnZ_dev) <= 1e-3, (lnZ, lnZ_dev)
    return heavy, exp_h, float(np.max(d_r)) if rest.size else 0.0


def high_snr_realisable(orc, snr=150.0):
    th_true = np.array([2.2, -0.5, 1.1, 0.7, 1.4, 300.0])
    probe = S.high_snr_problem(snr=snr, point=0)
    F, Y, _, dt = orc.coeffs(probe, th_true)
    return S.high_snr_problem(snr=snr, point=0, a0=np.outer(F[0], Y[0]), dt_true=dt[0])


def test_high_snr_mixed_full_size(G, orc):
    """SNR 150, RIFT_MIXED, 10 adaptive iterations of 1e6 samples (the high-SNR bench
    step); the weighted samples are float64 on the device, so they meet the oracle to 1e-6."""
    p = high_snr_realisable(orc)
    n = 1_000_000
    with G.ILE(p, precision=G.RIFT_MIXED, max_samples=n, n_bins=64, seed=1) as s:
        r = s.adapt(10, n)
        assert r["status"] == 0
        th, lr, ll, lw = s.last_batch(n)
    heavy, exp_h, d_rest = check_last_batch(orc, p, th, lr, ll, lw, r["lnZ_iter"][-1], all_bar=None)
    assert np.max(np.abs(ll[heavy] - exp_h)) <= 1e-6
    assert heavy.size >= 100
    print(f"SNR 150 mixed: {heavy.size} weighted samples to {np.max(np.abs(ll[heavy] - exp_h)):.1e}; "
          f"the float32 values of 300 others to {d_rest:.1e}")


def test_three_member_portfolio_full_size(G, orc):
    """The single large solve's portfolio of histogram, AV and Gaussian mixture at 1e6
    samples per iteration in float32 (the bench's portfolio block), four iterations."""
    p = S.single_large_problem()
    n = 1_000_000
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=n, n_bins=64, seed=1) as s:
        r = s.portfolio(4, n, members=G.RIFT_MEMBER_HIST | G.RIFT_MEMBER_AV | G.RIFT_MEMBER_GMM, p_thr=0.999,
                        n_min_star=1000, gmm_components=4, restart=True)
        assert r["status"] == 0
        info = s.portfolio_info()
        th, lr, ll, lw = s.last_batch(n)
    assert min(info["n_drawn"]) > 0
    check_last_batch(orc, p, th, lr, ll, lw, r["lnZ_iter"][-1])


def test_adaptive_volume_full_size(G, orc):
    """The adaptive-volume integrator at 1e6 samples per iteration in float32 on the single
    large solve, four iterations."""
    p = S.single_large_problem()
    n = 1_000_000
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=n, seed=1) as s:
        r = s.av(4, n, p_thr=0.999, n_min_star=1000, capacity=4 * n, restart=True)
        assert r["status"] == 0
        th, lr, ll, lw = s.last_batch(n)
    check_last_batch(orc, p, th, lr, ll, lw, r["lnZ_iter"][-1])
