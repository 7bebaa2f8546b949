"""Overlaps computed on the device (rift_ile_set_waveforms) against the oracle's
plain sums, and the likelihood built from them against the oracle's."""
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


def inputs(p):
    wf = p.meta["waveforms"]
    return wf.freqs, wf.h, p.meta["data"], wf.w


@pytest.mark.parametrize("which", ["plain", "large", "one_det"])
def test_overlaps_match_oracle(G, orc, which):
    from oracle import precompute as PC
    p = {"plain": S.plain_fp64_problem, "large": S.single_large_problem,
         "one_det": lambda: S.make_problem(("V1",), 7, 4096.0, n_t=401, snr=15.0, seed=S.config_seed(3, 77))}[which]()
    f, h, d, w = inputs(p)
    Q, U, V = PC.overlaps(f, h, d, w, p.q_t0, p.fs, p.n_q)
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=2000, set_overlaps=False) as s:
        s.set_waveforms(f, h, d, w)
        th = S.prior_samples(500, 5)
        got = s.eval(th)
        gQ, gU, gV = s.get_overlaps(p.n_q)
    qs, us, vs = np.max(np.abs(Q)), np.max(np.abs(U)), np.max(np.abs(V))
    assert np.max(np.abs(gQ - Q)) <= 1e-12 * qs
    assert np.max(np.abs(gU - U)) <= 1e-13 * us and np.max(np.abs(gV - V)) <= 1e-13 * vs
    assert np.array_equal(gU, np.conj(np.transpose(gU, (0, 2, 1))))   # mirrored exactly
    assert np.array_equal(gV, np.transpose(gV, (0, 2, 1)))
    # the likelihood from the device's overlaps against the oracle's on the oracle's
    op = S.Problem(p.det_names, p.det_tensor, p.det_pos, p.gmst, p.lm, p.fs, p.n_q, p.q_t0, Q, U, V, p.t_lo,
                   p.t_hi, p.n_t, p.d_ref, p.d_min, p.d_max, p.quad_norm)
    exp = orc.lnL(op, th)
    assert np.max(np.abs(got - exp) / np.maximum(1.0, np.abs(exp))) < 1e-9
    # and the oracle's overlaps agree with the generator's own (the same definition)
    assert np.max(np.abs(Q - p.Q)) <= 1e-10 * qs


def test_waveforms_device_inputs_and_errors(G, orc):
    import torch
    p = S.plain_fp64_problem()
    f, h, d, w = inputs(p)
    th = S.prior_samples(300, 8)
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=1000) as ref:
        exp = ref.eval(th)
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=1000, set_overlaps=False) as s:
        T = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (f, h, d, w)]
        s.set_waveforms(*T)
        got = s.eval(th)
        assert np.max(np.abs(got - exp) / np.maximum(1.0, np.abs(exp))) < 1e-9
        bad = f.copy()
        bad[0] += 1.0
        with pytest.raises(G.RiftError) as e:
            s.set_waveforms(bad, h, d, w)
        assert e.value.code == G.RIFT_EINVAL
        wb = w.copy()
        wb[0, 0] *= 2.0
        with pytest.raises(G.RiftError) as e:
            s.set_waveforms(f, h, d, wb)
        assert e.value.code == G.RIFT_EINVAL
        wb = w.copy()
        wb[0, 0] = wb[0, -1] = np.nan
        with pytest.raises(G.RiftError) as e:
            s.set_waveforms(f, h, d, wb)
        assert e.value.code == G.RIFT_ENONFINITE


def test_fft_and_direct_sum_agree_on_the_workload_grids(G, monkeypatch):
    """The workload grids lie on a lattice (+-2..256 Hz in steps of 2 Hz, f = 0 left out),
    so Q comes from the FFT path; forcing the direct sum gives the same Q to 1e-12 of
    max |Q|, and identical U, V."""
    for p in (S.plain_fp64_problem(), S.single_large_problem()):
        f, h, d, w = inputs(p)
        got = {}
        for dft in ("0", "1"):
            monkeypatch.setenv("RIFT_ILE_DFT", dft)
            with G.ILE(p, precision=G.RIFT_FP64, max_samples=16, set_overlaps=False) as s:
                s.set_waveforms(f, h, d, w)
                got[dft] = s.get_overlaps(p.n_q)
        (Qf, Uf, Vf), (Qd, Ud, Vd) = got["0"], got["1"]
        assert np.max(np.abs(Qf - Qd)) <= 1e-12 * np.max(np.abs(Qd))
        assert np.array_equal(Uf, Ud) and np.array_equal(Vf, Vd)


def long_segment_inputs(n_freq, df, K, M, seed, jitter=0.0):
    """A two-sided mirror-symmetric grid of n_freq frequencies (f_j = (j - (n_freq-1)/2) df,
    optionally moved off the lattice by a symmetric jitter), random mode waveforms and
    data, and symmetric weights."""
    rng = np.random.default_rng(seed)
    half = n_freq // 2
    fpos = (np.arange(half) + 0.5) * df
    if jitter:
        fpos = fpos + jitter * df * rng.random(half)
    f = np.concatenate([-fpos[::-1], fpos])
    h = (rng.normal(size=(M, n_freq)) + 1j * rng.normal(size=(M, n_freq))) / np.sqrt(n_freq)
    d = (rng.normal(size=(K, n_freq)) + 1j * rng.normal(size=(K, n_freq))) / np.sqrt(n_freq)
    wpos = rng.uniform(0.5, 2.0, size=(K, half))
    w = np.concatenate([wpos[:, ::-1], wpos], axis=1)
    return f, h, d, w


@pytest.mark.parametrize("jitter", [0.0, 0.3])
def test_long_segment_overlaps_against_oracle(G, jitter):
    """A 4 s segment at 4096 Hz: 2^14 frequencies (df = 0.25 Hz, L = f_s / df = 2^14).  On the
    lattice Q comes from the radix-2 FFT, off it (jitter) from the direct sum; both against
    the oracle's plain sums to 1e-12 of max |Q| (Eq. QUV), U and V to 1e-12 of their maxima."""
    from oracle import precompute as PC
    p = S.make_problem(("H1", "L1"), 4, 4096.0, n_t=401, snr=15.0, seed=S.config_seed(3, 81))
    f, h, d, w = long_segment_inputs(1 << 14, 0.25, p.n_det, p.n_modes, 17, jitter)
    Q, U, V = PC.overlaps(f, h, d, w, p.q_t0, p.fs, p.n_q)
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=16, set_overlaps=False) as s:
        s.set_waveforms(f, h, d, w)
        gQ, gU, gV = s.get_overlaps(p.n_q)
    assert np.max(np.abs(gQ - Q)) <= 1e-12 * np.max(np.abs(Q))
    assert np.max(np.abs(gU - U)) <= 1e-12 * np.max(np.abs(U))
    assert np.max(np.abs(gV - V)) <= 1e-12 * np.max(np.abs(V))
