"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, on the
same seeded inputs.

Tolerances:
  * RIFT_FP64 path: 1e-9 relative on every ln L value and on ln Z.
  * RIFT_FP32 path: |d ln L| <= 1e-3 on every sample (and every time bin), |d ln Z| <= 1e-3.
  * Integer and index work (sample streams, histogram bins) is compared exactly.
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


def rel(a, b):
    return np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b)))


FP32_TOL = 1e-3   # |d ln L| on every sample, and |d ln Z|, for the float32 path


def assert_fp32_close(got, exp, quad=None):
    """Float32 bar: |d ln L| <= 1e-3 on every sample.  (quad, the template term, is
    accepted for the callers' convenience; the bar does not depend on it.)"""
    got, exp = np.asarray(got), np.asarray(exp)
    d = np.abs(got - exp)
    assert np.max(d) <= FP32_TOL, (np.max(d), int(np.argmax(d)))


def olnL(orc, p, th):
    ll, _, quad = orc.lnL(p, th, want_bins=True) if len(th) <= 2000 else (None, None, None)
    if ll is None:
        ll = np.empty(len(th))
        quad = np.empty(len(th))
        for i in range(0, len(th), 2000):
            a, _, q = orc.lnL(p, th[i:i + 2000], want_bins=True)
            ll[i:i + 2000], quad[i:i + 2000] = a, q
    return ll, quad


# ------------------------------------------------------------------------------ FP64 plain path

def test_fp64_coeffs_match_oracle(G, orc):
    p = S.single_large_problem()
    th = S.prior_samples(500, 31)
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=1000) as s:
        c, dt, quad = s.coeffs(th)
    _, _, oc, odt = orc.coeffs(p, th)
    _, _, oquad = orc.lnL(p, th, want_bins=True)
    assert np.max(np.abs(c - oc)) < 1e-12 * max(1.0, np.max(np.abs(oc)))
    assert np.max(np.abs(dt - odt)) < 1e-15
    assert rel(quad, oquad) < 1e-11


def test_fp64_eval_plain_config(G, orc):
    """Two detectors, modes (2,+-2), 401 bins: every sample and every bin."""
    p = S.plain_fp64_problem()
    th = S.prior_samples(10000, 32)
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=4096) as s:
        got = s.eval(th)
        gb, gbins = s.eval(th[:300], want_bins=True)
    exp = orc.lnL(p, th)
    assert rel(got, exp) < 1e-9
    eb, ebins, _ = orc.lnL(p, th[:300], want_bins=True)
    assert rel(gbins, ebins) < 1e-9
    assert np.array_equal(gb, got[:300])


def test_fp64_eval_all_modes(G, orc):
    p = S.single_large_problem()
    th = S.prior_samples(700, 33)
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=256) as s:
        got, gbins = s.eval(th, want_bins=True)
    exp, ebins, _ = orc.lnL(p, th, want_bins=True)
    assert rel(got, exp) < 1e-9
    assert rel(gbins, ebins) < 1e-9


def test_fp64_marginalize_same_stream_as_oracle(G, orc):
    """The device's Philox stream and inverse-CDF draw equal the oracle's; the
    histogram bins and ln p - ln p_s agree exactly; ln Z to 1e-9."""
    p = S.plain_fp64_problem()
    n = 10000
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=n, n_bins=32, seed=1234) as s:
        r = s.marginalize(n)
        th, lr, ll, lw = s.last_batch(n)
    sm = orc.Sampler(n_bins=32, seed=1234)
    oth, olr, obins = sm.draw(n)
    assert np.max(np.abs(th - oth)) < 1e-12
    assert np.array_equal(lr, olr)
    oll = orc.lnL(p, oth)
    assert rel(ll, oll) < 1e-9
    red = orc.reduce(oll + olr)
    assert abs(r["lnZ"] - red["lnZ"]) < 1e-9 * max(1, abs(red["lnZ"]))
    assert abs(r["n_eff"] - red["n_eff"]) < 1e-9 * red["n_eff"]
    assert abs(r["n_ess"] - red["n_ess"]) < 1e-9 * red["n_ess"]
    assert abs(r["sigma_lnZ"] - red["sigma_lnZ"]) < 1e-9


def test_fp64_adapt_matches_oracle_loop(G, orc):
    """Three adaptive iterations: per-iteration ln Z, pooled ln Z and the
    adapted histogram masses follow the oracle's loop."""
    p = S.plain_fp64_problem()
    n, iters = 20000, 3
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=n, n_bins=24, seed=99, adapt_floor=0.1) as s:
        r = s.adapt(iters, n)
        P = s.sampler()
    sm = orc.Sampler(n_bins=24, seed=99, floor=0.1)
    ref = orc.run_adapt(p, sm, iters, n)
    for g in range(iters):
        assert abs(r["lnZ_iter"][g] - ref["iterations"][g]["lnZ"]) < 1e-9 * max(1, abs(ref["iterations"][g]["lnZ"]))
    assert abs(r["lnZ"] - ref["pooled"]["lnZ"]) < 1e-9 * max(1, abs(ref["pooled"]["lnZ"]))
    assert abs(r["n_eff"] - ref["pooled"]["n_eff"]) < 1e-8 * ref["pooled"]["n_eff"]
    assert r["n_total"] == n * iters
    # masses agree to the rounding of weighted sums with a wide dynamic range
    assert np.max(np.abs(P - sm.P)) < 1e-10


# ------------------------------------------------------------------------------ FP32 path

@pytest.mark.parametrize("n", [1, 63, 64, 65, 3001])
def test_fp32_eval_sizes_single_large(G, orc, n):
    """21 modes, 3 detectors, 1001 bins; sizes across tile boundaries and a ragged tail."""
    p = S.single_large_problem()
    th = S.prior_samples(n, 40 + n)
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=4096) as s:
        got = s.eval(th)
    assert_fp32_close(got, *olnL(orc, p, th))


def test_fp32_bins_match(G, orc):
    p = S.single_large_problem()
    th = S.prior_samples(200, 41)
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=4096) as s:
        got, gbins = s.eval(th, want_bins=True)
    exp, ebins, quad = orc.lnL(p, th, want_bins=True)
    assert np.max(np.abs(gbins - ebins)) <= FP32_TOL, np.max(np.abs(gbins - ebins))
    assert_fp32_close(got, exp, quad)


def test_fp32_plain_config_and_batching(G, orc):
    """Few modes, and n above max_samples (the call processes several batches)."""
    p = S.plain_fp64_problem()
    th = S.prior_samples(5000, 42)
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=1024) as s:
        got = s.eval(th)
    assert_fp32_close(got, *olnL(orc, p, th))


def test_fp32_unsorted_sky_and_polar_caps(G, orc):
    """Samples spread over the whole sky in one batch (tiles straddling cells),
    plus samples near the poles and at alpha = 0 / 2 pi."""
    p = S.single_large_problem()
    th = S.prior_samples(1500, 43)
    th[:200, 1] = np.sign(th[:200, 1]) * (math.pi / 2 - np.abs(th[:200, 1]) * 1e-3)
    th[200:300, 0] = np.where(np.arange(100) % 2, 1e-9, 2 * math.pi - 1e-9)
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=4096) as s:
        got = s.eval(th)
    assert_fp32_close(got, *olnL(orc, p, th))


def test_fp32_device_memory_inputs(G, orc):
    import torch
    p = S.single_large_problem()
    th = S.prior_samples(777, 44)
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=512) as s:
        tt = torch.from_numpy(th).cuda()
        got = s.eval(tt).cpu().numpy()
        got_host = s.eval(th)
    assert_fp32_close(got, *olnL(orc, p, th))
    assert np.max(np.abs(got - got_host)) <= 1e-6 * np.max(np.abs(got))


def test_fp32_marginalize_against_oracle_on_device_stream(G, orc):
    """ln Z of one batch: the oracle re-evaluates the device's own theta stream."""
    p = S.single_large_problem()
    n = 20000
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=n, n_bins=32, seed=5) as s:
        r = s.marginalize(n)
        th, lr, ll, lw = s.last_batch(n)
    oll, oq = olnL(orc, p, th)
    assert_fp32_close(ll, oll, oq)
    red = orc.reduce(oll + lr)
    assert abs(r["lnZ"] - red["lnZ"]) <= 1e-3
    assert abs(r["n_eff"] - red["n_eff"]) <= 1e-2 * red["n_eff"]


def test_fp32_reduction_against_float64_reduction_of_same_weights(G, orc):
    """The float32 path sums float32 exponentials of ln w - max.  The oracle's float64
    reduction of the device's own ln w pins that reduction alone: the terms' ~1e-7
    relative error moves ln Z and n_eff by far less than the float32 bars."""
    p = S.single_large_problem()
    n = 50000
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=n, n_bins=32, seed=12) as s:
        r = s.marginalize(n)
        th, lr, ll, lw = s.last_batch(n)
    red = orc.reduce(lw)
    assert abs(r["lnZ"] - red["lnZ"]) <= 1e-6
    assert abs(r["n_eff"] - red["n_eff"]) <= 1e-6 * red["n_eff"]
    assert abs(r["n_ess"] - red["n_ess"]) <= 1e-6 * red["n_ess"]


@pytest.mark.parametrize("tc", ["0", "1"])
def test_fp32_adapt_two_iterations(G, orc, monkeypatch, tc):
    """Adaptive iterations through the CUDA-core and the tensor-core kernels.  The
    batch's ln L must be the float32 kernel's own output: it differs from the
    float64 kernel's values in the low bits of (almost) every sample."""
    monkeypatch.setenv("RIFT_ILE_TC", tc)
    p = S.single_large_problem()
    n = 30000
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=n, n_bins=32, seed=6) as s:
        r = s.adapt(2, n)
        th, lr, ll, lw = s.last_batch(n)
    oll = orc.lnL(p, th)
    red = orc.reduce(oll + lr)
    assert abs(r["lnZ_iter"][1] - red["lnZ"]) <= 1e-3
    assert r["n_total"] == 2 * n
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=n) as s64:
        ll64 = s64.eval(th)
    assert np.mean(ll == ll64) < 0.05


# ------------------------------------------------------------------------------ tensor-core tiles

def clustered_samples(n, seed, center=(1.0, 0.3), width=0.06):
    """Prior draws with the sky confined to a small patch, so that 128-sample
    tiles share narrow Q windows even in a small batch."""
    th = S.prior_samples(n, seed)
    rng = np.random.default_rng(seed + 1)
    th[:, 0] = center[0] + width * rng.random(n)
    th[:, 1] = center[1] + width * rng.random(n)
    return th


@pytest.mark.parametrize("n", [1, 127, 128, 129, 6000])
def test_tc_path_matches_oracle(G, orc, monkeypatch, n):
    """The tcgen05 contraction (float16 hi/lo split, 3 MMAs per K step) against
    the oracle, at sizes across the 128-sample tile and a ragged tail."""
    monkeypatch.setenv("RIFT_ILE_TC", "1")
    p = S.single_large_problem()
    th = clustered_samples(n, 61 + n)
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=8192) as s:
        got = s.eval(th)
    assert_fp32_close(got, *olnL(orc, p, th))


def test_tc_path_bins_and_cuda_core_agree(G, orc, monkeypatch):
    p = S.single_large_problem()
    th = clustered_samples(700, 62)
    monkeypatch.setenv("RIFT_ILE_TC", "1")
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=1024) as s:
        g_tc, b_tc = s.eval(th, want_bins=True)
    monkeypatch.setenv("RIFT_ILE_TC", "0")
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=1024) as s:
        g_cc, b_cc = s.eval(th, want_bins=True)
    exp, ebins, quad = orc.lnL(p, th, want_bins=True)
    assert np.max(np.abs(b_tc - ebins)) <= FP32_TOL
    assert_fp32_close(g_tc, exp, quad)
    assert_fp32_close(g_cc, exp, quad)
    # two float32 evaluations, each within the float32 bar of the oracle, agree within the
    # sum of their bars
    assert np.max(np.abs(g_tc - g_cc)) <= 2 * FP32_TOL


def test_tc_path_plain_config_and_spread_sky(G, orc, monkeypatch):
    """Two modes (K padded to 16) and an unclustered sky (wide tiles take the
    direct fallback inside the tensor kernel)."""
    monkeypatch.setenv("RIFT_ILE_TC", "1")
    for p, th in ((S.plain_fp64_problem(), clustered_samples(3000, 63)),
                  (S.single_large_problem(), S.prior_samples(3000, 64))):
        with G.ILE(p, precision=G.RIFT_FP32, max_samples=4096) as s:
            got = s.eval(th)
        assert_fp32_close(got, *olnL(orc, p, th))


# ------------------------------------------------------------------------------ mixed precision

def high_snr_realisable(orc, snr=150.0, seed=71):
    """21 modes, 3 detectors, 16384 Hz, q=20-like hierarchy, an injection built
    from F_k Y_lm at theta_true (so ln L reaches ~snr^2/2 near theta_true)."""
    th_true = np.array([2.2, -0.5, 1.1, 0.7, 1.4, 300.0])
    probe = S.high_snr_problem(snr=snr, point=seed)
    F, Y, _, dt = orc.coeffs(probe, th_true)
    p = S.high_snr_problem(snr=snr, point=seed, a0=np.outer(F[0], Y[0]), dt_true=dt[0])
    return p, th_true


def test_mixed_precision_high_snr(G, orc):
    """SNR 150: samples near the injection have ln L ~ 1e4.  The float32 path
    carries ~1e-3..1e-2 rounding there; RIFT_MIXED re-evaluates every sample
    within 40 of the batch maximum in float64 and meets 1e-3."""
    p, th_true = high_snr_realisable(orc)
    rng = np.random.default_rng(8)
    near = th_true + rng.normal(0, 1, (600, 6)) * np.array([6e-4, 6e-4, 1.5e-3, 1.5e-3, 1.5e-3, 0.3])
    th = np.concatenate([near, S.prior_samples(1400, 72)])
    exp, _, quad = orc.lnL(p, th, want_bins=True)
    assert exp.max() > 5000
    with G.ILE(p, precision=G.RIFT_MIXED, max_samples=4096) as s:
        got = s.eval(th)
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=4096) as s:
        got32 = s.eval(th)
    top = exp >= exp.max() - 40.0
    assert top.sum() >= 50
    assert np.max(np.abs(got[top] - exp[top])) <= 1e-3
    assert_fp32_close(got, exp)
    # the float32 path alone is measurably worse on the same samples
    assert np.max(np.abs(got32[top] - exp[top])) > np.max(np.abs(got[top] - exp[top]))


def test_mixed_precision_reproducible(G, orc):
    """RIFT_MIXED twice on the same seed: the selection of the samples to re-evaluate is
    in index order and the float32 bins come from fixed tiles, so every value repeats
    exactly."""
    p, _ = high_snr_realisable(orc)
    n = 20000
    out = []
    for _ in range(2):
        with G.ILE(p, precision=G.RIFT_MIXED, max_samples=n, n_bins=32, seed=11) as s:
            r = s.adapt(2, n)
            out.append((r, s.last_batch(n)))
    (r0, b0), (r1, b1) = out
    assert r0["lnZ_iter"] == r1["lnZ_iter"] and r0["lnZ"] == r1["lnZ"]
    for a, b in zip(b0, b1):
        assert np.array_equal(a, b)


def test_mixed_precision_adapt_lnZ(G, orc):
    """Adaptive iterations in RIFT_MIXED at SNR 150: ln Z of the device's own
    sample stream within 1e-3 of the oracle's."""
    p, th_true = high_snr_realisable(orc)
    n = 20000
    with G.ILE(p, precision=G.RIFT_MIXED, max_samples=n, n_bins=32, seed=9) as s:
        r = s.adapt(3, n)
        th, lr, ll, lw = s.last_batch(n)
    oll, oq = olnL(orc, p, th)
    red = orc.reduce(oll + lr)
    assert abs(r["lnZ_iter"][2] - red["lnZ"]) <= 1e-3
    top = oll + lr >= np.max(oll + lr) - 40.0
    assert np.max(np.abs(ll[top] - oll[top])) <= 1e-3


# ------------------------------------------------------------------------------ full size

@pytest.mark.slow
def test_full_size_single_large_every_sample(G, orc):
    """1e6 samples, 3 detectors, 21 modes, 1001 bins, the benchmark's launch
    configuration (an adapted sampling prior, then one batch): every one of the 1e6
    ln L values against the oracle's, and ln Z against the oracle's reduction of the
    oracle's own ln L on the device's sample stream."""
    p = S.single_large_problem()
    n = 1_000_000
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=n, n_bins=64, seed=7) as s:
        s.adapt(1, n)
        r = s.marginalize(n)
        th, lr, ll, lw = s.last_batch(n)
    oll = orc.lnL(p, th)
    d = np.abs(ll - oll)
    print(f"full size: max |d ln L| over {n} samples = {d.max():.3e}")
    assert np.max(d) <= FP32_TOL, (np.max(d), int(np.argmax(d)))
    red = orc.reduce(oll + lr)
    assert abs(r["lnZ"] - red["lnZ"]) <= FP32_TOL, (r["lnZ"], red["lnZ"])
    assert r["n_total"] == n


# ------------------------------------------------------------------------------ edges and state

def test_empty_and_errors(G):
    p = S.plain_fp64_problem()
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=100) as s:
        out = s.eval(np.zeros((0, 6)))
        assert out.shape == (0,)
        with pytest.raises(G.RiftError) as e:
            s.marginalize(101)
        assert e.value.code == G.RIFT_EINVAL
        with pytest.raises(G.RiftError) as e:
            s.adapt(0, 10)
        assert e.value.code == G.RIFT_EINVAL
        Qbad = p.Q.copy()
        Qbad[0, 0, 5] = np.nan
        with pytest.raises(G.RiftError) as e:
            s.set_overlaps(Qbad, p.U, p.V)
        assert e.value.code == G.RIFT_ENONFINITE
        Ubad = p.U.copy()
        Ubad[0, 0, 1] += 1.0
        with pytest.raises(G.RiftError) as e:
            s.set_overlaps(p.Q, Ubad, p.V)
        assert e.value.code == G.RIFT_EINVAL


def test_no_overlaps_is_state_error(G):
    p = S.plain_fp64_problem()
    s = G.ILE(p, precision=G.RIFT_FP32, max_samples=100, set_overlaps=False)
    with pytest.raises(G.RiftError) as e:
        s.eval(S.prior_samples(3, 1))
    assert e.value.code == G.RIFT_ESTATE
    s.close()


def test_checkpoint_resume_reproduces_stream(G):
    """get_state after one adaptation, then: continuing, and restoring the
    state in a fresh handle, give the same next batch."""
    p = S.plain_fp64_problem()
    n = 5000
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=n, n_bins=16, seed=11) as a:
        a.adapt(1, n)
        blob = a.get_state()
        ra = a.marginalize(n)
        tha = a.last_batch(n)[0]
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=n, n_bins=16, seed=999) as b:
        b.set_state(blob)
        rb = b.marginalize(n)
        thb = b.last_batch(n)[0]
        with pytest.raises(G.RiftError):
            b.set_state(blob[:-8])
    assert np.array_equal(tha, thb)
    assert ra["lnZ"] == rb["lnZ"]


def test_quad_norm_half_with_half_grams(G):
    p = S.plain_fp64_problem()
    th = S.prior_samples(300, 50)
    import copy
    h = copy.copy(p)
    h.quad_norm = 1
    h.U, h.V = p.U / 2, p.V / 2
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=512) as a, G.ILE(h, precision=G.RIFT_FP64, max_samples=512) as b:
        assert rel(a.eval(th), b.eval(th)) < 1e-11


def test_bounded_wait_reports_timeout_and_context_survives(G):
    """The tensor-core kernels' bounded wait, run on a barrier nothing completes, gives up
    after its limit, the call returns RIFT_ETIMEOUT, and the handle keeps working."""
    import time
    p = S.plain_fp64_problem()
    th = S.prior_samples(200, 3)
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=256) as s:
        before = s.eval(th)
        t0 = time.perf_counter()
        rc = G.rift_ile_wait_selftest(s.h, 20_000_000)   # 20 ms
        dt = time.perf_counter() - t0
        assert rc == G.RIFT_ETIMEOUT
        assert dt >= 0.02
        assert G.rift_ile_wait_selftest(s.h, 10) == G.RIFT_EINVAL
        after = s.eval(th)
    assert np.array_equal(before, after)


@pytest.mark.parametrize("delay3", ["0", "1"])
def test_tc_path_three_detector_sort_keys(G, orc, monkeypatch, delay3):
    """Three detectors sorted by the sky curve or by a Morton key of their three delays:
    the same float32 results within the bar, through eval and through adaptation."""
    monkeypatch.setenv("RIFT_ILE_TC", "1")
    monkeypatch.setenv("RIFT_ILE_DELAY3", delay3)
    p = S.single_large_problem()
    th = S.prior_samples(1500, 91)
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=20000, n_bins=32, seed=19) as s:
        got = s.eval(th)
        r = s.adapt(2, 20000)
        bth, lr, ll, lw = s.last_batch(20000)
    assert_fp32_close(got, *olnL(orc, p, th))
    red = orc.reduce(orc.lnL(p, bth) + lr)
    assert abs(r["lnZ_iter"][1] - red["lnZ"]) <= 1e-3
