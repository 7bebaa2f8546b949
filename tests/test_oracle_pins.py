"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test names the part of the oracle it pins and the reason a plausible slip
(dropped term, wrong sign, wrong index, transposed operand) would fail it.
CPU only.
"""
import copy
import math

import numpy as np
import pytest

import ile_synth as S


@pytest.fixture(scope="module")
def orc(oracle_lib):
    return oracle_lib


def _grid_time(p, j):
    return p.t_lo + j * (p.t_hi - p.t_lo) / (p.n_t - 1)


def _regrid(p, t0):
    """Same data, Q re-evaluated (by definition) on grids starting at t0[k]."""
    q = copy.copy(p)
    q.q_t0 = np.asarray(t0, float)
    wf = p.meta["waveforms"]
    rng = np.random.default_rng(p.meta["seed"] + 7919)
    Q = np.zeros_like(p.Q)
    data = []
    for k in range(p.n_det):
        d = wf.strain(p.meta["a_true"][k], p.meta["t_true"] + p.meta["dt_true"][k])
        if p.meta["noise"]:
            d = d + wf.noise(k, rng)
        data.append(d)
        Q[k] = wf.overlap_series(k, d, q.q_t0[k] + np.arange(p.n_q) / p.fs)
    q.Q = Q
    return q, data


# ---- P6: spin-weighted harmonics ---------------------------------------------------------

@pytest.mark.parametrize("iota,phi", [(0.3, 0.1), (1.2, -2.0), (2.9, 4.0), (0.0, 0.5), (math.pi, 1.0)])
def test_p6_l2_closed_forms(orc, iota, phi):
    """-2Y_2m against the textbook closed forms (a wrong factorial, power or
    sign in the Wigner-d sum fails at least one m)."""
    c, s = math.cos(iota), math.sin(iota)
    exp = {
        2: math.sqrt(5 / (64 * math.pi)) * (1 + c) ** 2,
        1: math.sqrt(5 / (16 * math.pi)) * s * (1 + c),
        0: math.sqrt(15 / (32 * math.pi)) * s * s,
        -1: math.sqrt(5 / (16 * math.pi)) * s * (1 - c),
        -2: math.sqrt(5 / (64 * math.pi)) * (1 - c) ** 2,
    }
    for m, a in exp.items():
        assert abs(orc.sYlm(2, m, iota, phi) - a * np.exp(1j * m * phi)) < 1e-14


def test_p6_orthonormality(orc):
    """Integral of Y_lm conj(Y_l'm') over the sphere is the identity for all
    21 modes with 2 <= l <= 4 (Gauss-Legendre in cos(theta) x uniform phi)."""
    x, w = np.polynomial.legendre.leggauss(24)
    nphi = 16
    phis = 2 * np.pi * np.arange(nphi) / nphi
    modes = S.MODE_ORDER
    Y = np.array([[[orc.sYlm(l, m, math.acos(xx), ph) for ph in phis] for xx in x] for (l, m) in modes])
    G = np.einsum("aij,bij,i->ab", Y, np.conj(Y), w) * (2 * np.pi / nphi)
    assert np.max(np.abs(G - np.eye(len(modes)))) < 1e-12


def test_p6_reflection_symmetry(orc):
    """-2Y_l,-m(theta, phi) = (-1)^l conj(-2Y_lm(pi - theta, phi)) for l <= 4:
    the reflection identity of the Wigner-d functions (checked against the
    l = 2 closed forms above), which fails for a wrong sign of k or m in the sum."""
    for l in (2, 3, 4):
        for m in range(-l, l + 1):
            for iota in (0.4, 1.9):
                lhs = orc.sYlm(l, -m, iota, 0.7)
                rhs = (-1) ** l * np.conj(orc.sYlm(l, m, math.pi - iota, 0.7))
                assert abs(lhs - rhs) < 1e-14


# ---- P7 / P8: detector response and delays ---------------------------------------------

def test_p7_response_thorne_closed_form(orc):
    """Arms along x and y, gmst = 0: F_+ and F_x against the detector-frame
    closed forms with source polar angle th = pi/2 - delta and azimuth alpha:
      F_+ = 1/2 (1 + cos^2 th) cos 2a cos 2psi - cos th sin 2a sin 2psi
      F_x = 1/2 (1 + cos^2 th) cos 2a sin 2psi + cos th sin 2a cos 2psi
    The sky basis used here measures psi from the other axis and in the other
    sense, so the textbook angle is pi/2 - psi; with that map both components
    agree exactly (a wrong basis vector or a sign in F_x breaks it)."""
    D = 0.5 * (np.outer([1, 0, 0], [1, 0, 0]) - np.outer([0, 1, 0], [0, 1, 0]))
    rng = np.random.default_rng(4)
    for _ in range(50):
        a, d, psi = rng.uniform(0, 2 * np.pi), rng.uniform(-1.5, 1.5), rng.uniform(0, np.pi)
        th = math.pi / 2 - d
        fp, fx = orc.antenna(D, a, d, psi, 0.0)
        p = math.pi / 2 - psi
        ep = 0.5 * (1 + math.cos(th) ** 2) * math.cos(2 * a) * math.cos(2 * p) - math.cos(th) * math.sin(2 * a) * math.sin(2 * p)
        ex = 0.5 * (1 + math.cos(th) ** 2) * math.cos(2 * a) * math.sin(2 * p) + math.cos(th) * math.sin(2 * a) * math.cos(2 * p)
        assert abs(fp - ep) < 1e-13 and abs(fx - ex) < 1e-13


def test_p7_response_invariants(orc):
    """|F|^2 is psi-independent; F(psi + pi/2) = -F(psi); the wave is
    transverse (D = s s^T gives F = 0)."""
    tens, _ = S.detector_geometry("L1")
    rng = np.random.default_rng(5)
    for _ in range(30):
        a, d, g = rng.uniform(0, 2 * np.pi), rng.uniform(-1.5, 1.5), rng.uniform(0, 2 * np.pi)
        vals = [orc.antenna(tens, a, d, psi, g) for psi in (0.1, 0.8, 2.5)]
        n2 = [x * x + y * y for x, y in vals]
        assert max(n2) - min(n2) < 1e-14
        f0 = orc.antenna(tens, a, d, 0.3, g)
        f1 = orc.antenna(tens, a, d, 0.3 + math.pi / 2, g)
        assert abs(f0[0] + f1[0]) < 1e-14 and abs(f0[1] + f1[1]) < 1e-14
        s = np.array([math.cos(d) * math.cos(a - g), math.cos(d) * math.sin(a - g), math.sin(d)])
        fz = orc.antenna(np.outer(s, s), a, d, 0.3, g)
        assert abs(fz[0]) < 1e-14 and abs(fz[1]) < 1e-14


def test_p8_delay_bounds(orc):
    """|dt_k - dt_k'| <= |x_k - x_k'|/c, with equality along the baseline; a
    source over a detector's vertex arrives |x|/c before the geocentre."""
    _, xh = S.detector_geometry("H1")
    _, xl = S.detector_geometry("L1")
    base = np.linalg.norm(xh - xl) / S.C_SI
    rng = np.random.default_rng(6)
    for _ in range(200):
        a, d = rng.uniform(0, 2 * np.pi), math.asin(rng.uniform(-1, 1))
        assert abs(orc.delay(xh, a, d, 0.4) - orc.delay(xl, a, d, 0.4)) <= base * (1 + 1e-12)
    b = (xh - xl) / np.linalg.norm(xh - xl)
    d, a = math.asin(b[2]), math.atan2(b[1], b[0]) + 0.4
    assert abs((orc.delay(xl, a, d, 0.4) - orc.delay(xh, a, d, 0.4)) - base) < 1e-15
    u = xh / np.linalg.norm(xh)
    assert abs(orc.delay(xh, math.atan2(u[1], u[0]) + 0.4, math.asin(u[2]), 0.4)
               + np.linalg.norm(xh) / S.C_SI) < 1e-15


# ---- the decomposed likelihood vs the direct strain likelihood ---------------------------

def test_p5_decomposition_equals_direct_strain_likelihood(orc):
    """At a bin whose detector arrival times fall on Q samples, the oracle's
    ln L (Eq. def:lnL:Decomposed with kappa = 1/4) equals
    sum_k <h_k|d_k> - 1/2 <h_k|h_k> with h_k = Re sum_lm c_k,lm h_lm computed
    straight from the frequency-domain waveforms.  A wrong conjugate, a missing
    Re, V vs conj(V), the 1/4, or a transposed U all break this identity."""
    p = S.make_problem(("H1", "L1", "V1"), 9, 4096.0, n_t=401, snr=15.0, noise=True, seed=3)
    wf = p.meta["waveforms"]
    th = S.prior_samples(4, 11)
    _, _, c, dt = orc.coeffs(p, th)
    for i in range(4):
        j = 50 + 70 * i
        tj = _grid_time(p, j)
        q, data = _regrid(p, [tj + dt[i, k] - 300 / p.fs for k in range(3)])
        _, bins, _ = orc.lnL(q, th[i:i + 1], want_bins=True)
        exp = 0.0
        for k in range(3):
            h = wf.strain(c[i, k], tj + dt[i, k])
            exp += np.real(wf.inner(k, h, data[k])) - 0.5 * np.real(wf.inner(k, h, h))
        assert abs(bins[0, j] - exp) < 1e-11 * max(1.0, abs(exp))


def _realisable(orc, snr=20.0, noise=False, seed=21, n_modes=9):
    """A noise-free injection generated from F_k Y_lm at theta_true, with Q
    grids aligned so that t_true + dt_k falls on a Q sample."""
    th_true = np.array([1.1, 0.4, 0.7, 2.1, 1.0, 400.0])
    probe = S.make_problem(("H1", "L1", "V1"), n_modes, 4096.0, n_t=401, snr=snr, noise=noise, seed=seed)
    F, Y, _, dt = orc.coeffs(probe, th_true)
    a0 = np.outer(F[0], Y[0])
    j_true = 200
    t_true = _grid_time(probe, j_true)
    t0 = [t_true + dt[0, k] - 400 / probe.fs for k in range(3)]
    p = S.make_problem(("H1", "L1", "V1"), n_modes, 4096.0, n_t=401, snr=snr, noise=noise, seed=seed,
                       a0=a0, dt_true=dt[0], t_true=t_true, d_true=th_true[5], gmst=probe.gmst, q_t0=t0)
    return p, th_true, j_true


def test_p5_injection_peak_is_half_rho_squared(orc):
    """Noise-free consistent injection: ln L(theta_true, t_true) = rho^2/2
    exactly, and theta_true is a local maximum."""
    p, th_true, j = _realisable(orc)
    _, bins, _ = orc.lnL(p, th_true, want_bins=True)
    assert abs(bins[0, j] - 0.5 * p.meta["snr"] ** 2) < 1e-10 * p.meta["snr"] ** 2
    assert np.argmax(bins[0]) == j
    rng = np.random.default_rng(3)
    pert = th_true + rng.normal(0, 1e-3, (64, 6)) * np.array([1, 1, 1, 1, 1, 100.0])
    _, bp, _ = orc.lnL(p, pert, want_bins=True)
    assert np.all(bp[:, j] < bins[0, j])


def test_p4_quadratic_in_inverse_distance(orc):
    """ln L_j(x) with x = D_ref/D is exactly A x - B x^2, so its maximum sits at
    x* = A / 2B; a 3-point fit with a free constant returns C = 0 and predicts
    a 4th distance."""
    p = S.plain_fp64_problem()
    th = S.prior_samples(3, 8)
    for i in range(3):
        xs, vals = [], []
        for D in (150.0, 300.0, 600.0, 900.0):
            t = th[i].copy()
            t[5] = D
            _, b, _ = orc.lnL(p, t, want_bins=True)
            xs.append(p.d_ref / D)
            vals.append(b[0])
        xs, vals = np.array(xs), np.array(vals)
        A = np.stack([xs[:3], -xs[:3] ** 2, np.ones(3)], 1)
        sol = np.linalg.solve(A, vals[:3])
        assert np.max(np.abs(sol[2])) < 1e-9 * np.max(np.abs(vals))
        pred = sol[0] * xs[3] - sol[1] * xs[3] ** 2
        assert np.max(np.abs(pred - vals[3])) < 1e-9 * np.max(np.abs(vals))
        assert np.all(sol[1] > 0)


# ---- P1 / P2 / P3: symmetries and the template term --------------------------------------

def test_p1_psi_plus_pi(orc):
    p = S.single_large_problem()
    th = S.prior_samples(20, 9)
    a = orc.lnL(p, th)
    t2 = th.copy()
    t2[:, 2] += math.pi
    assert np.max(np.abs(orc.lnL(p, t2) - a)) < 1e-11 * max(1, np.max(np.abs(a)))


def test_p2_quadrupole_phase_symmetries(orc):
    """(2,+-2) only: phi -> phi + pi leaves ln L unchanged, and so does
    (psi, phi) -> (psi + pi/2, phi + pi/2) (F -> -F, Y_2+-2 -> -Y_2+-2).
    With odd-m modes present phi -> phi + pi must change ln L."""
    p = S.plain_fp64_problem()
    th = S.prior_samples(20, 10)
    a = orc.lnL(p, th)
    t2 = th.copy()
    t2[:, 3] += math.pi
    assert np.max(np.abs(orc.lnL(p, t2) - a)) < 1e-11 * np.max(np.abs(a))
    t3 = th.copy()
    t3[:, 2] += math.pi / 2
    t3[:, 3] += math.pi / 2
    assert np.max(np.abs(orc.lnL(p, t3) - a)) < 1e-11 * np.max(np.abs(a))
    p3 = S.make_problem(("H1", "L1"), 4, 4096.0, seed=12)
    b = orc.lnL(p3, th)
    assert np.max(np.abs(orc.lnL(p3, t2) - b)) > 1e-3


def test_p3_gram_inputs_and_nonnegative_template(orc):
    """U Hermitian, V symmetric; the template term is real and >= 0 for every
    sample (with Q = 0, ln L_j = -quad <= 0 at every bin)."""
    p = S.single_large_problem()
    for k in range(p.n_det):
        assert np.max(np.abs(p.U[k] - p.U[k].conj().T)) < 1e-12 * np.max(np.abs(p.U[k]))
        assert np.max(np.abs(p.V[k] - p.V[k].T)) < 1e-12 * np.max(np.abs(p.V[k]))
    z = copy.copy(p)
    z.Q = np.zeros_like(p.Q)
    th = S.prior_samples(200, 13)
    ll, bins, quad = orc.lnL(z, th, want_bins=True)
    assert np.all(quad >= 0)
    assert np.all(np.abs(bins + quad[:, None]) == 0)


def test_template_term_equals_half_signal_norm(orc):
    """quad(c) = 1/2 sum_k <h_k|h_k> for h_k = Re sum c h_lm, from waveforms."""
    p = S.make_problem(("H1", "L1", "V1"), 21, 4096.0, snr=10.0, seed=14)
    wf = p.meta["waveforms"]
    th = S.prior_samples(5, 15)
    _, _, c, _ = orc.coeffs(p, th)
    _, _, quad = orc.lnL(p, th, want_bins=True)
    for i in range(5):
        exp = sum(0.5 * np.real(wf.inner(k, wf.strain(c[i, k]), wf.strain(c[i, k]))) for k in range(3))
        assert abs(quad[i] - exp) < 1e-11 * exp


def test_quad_norm_half_matches_quarter_with_rescaled_grams(orc):
    """The 1/2 normalisation with (U, V)/2 reproduces the paper's 1/4 form."""
    p = S.plain_fp64_problem()
    th = S.prior_samples(10, 16)
    a = orc.lnL(p, th)
    h = copy.copy(p)
    h.quad_norm = 1
    h.U = p.U / 2
    h.V = p.V / 2
    assert np.max(np.abs(orc.lnL(h, th) - a)) < 1e-11 * np.max(np.abs(a))


# ---- P11 / P12: time marginalisation and interpolation ----------------------------------

def test_p12_interpolation_exact_for_linear_q(orc):
    """Q linear in time is reproduced exactly by the interpolation at any
    shifted time; the shift itself comes from the oracle's delays."""
    p = copy.copy(S.make_problem(("H1", "L1"), 3, 4096.0, seed=17))
    rng = np.random.default_rng(1)
    A = rng.normal(size=(2, 3)) + 1j * rng.normal(size=(2, 3))
    Bc = rng.normal(size=(2, 3)) + 1j * rng.normal(size=(2, 3))
    ts = [p.q_t0[k] + np.arange(p.n_q) / p.fs for k in range(2)]
    p.Q = np.stack([A[k][:, None] + Bc[k][:, None] * ts[k][None, :] for k in range(2)])
    p.U = np.zeros_like(p.U)
    p.V = np.zeros_like(p.V)
    th = S.prior_samples(5, 18)
    _, _, c, dt = orc.coeffs(p, th)
    _, bins, _ = orc.lnL(p, th, want_bins=True)
    tj = p.t_lo + np.arange(p.n_t) * (p.t_hi - p.t_lo) / (p.n_t - 1)
    for i in range(5):
        exp = sum(np.real(np.sum(np.conj(c[i, k])[:, None] * (A[k][:, None] + Bc[k][:, None] * (tj + dt[i, k])[None, :]), 0))
                  for k in range(2))
        assert np.max(np.abs(bins[i] - exp)) < 1e-10


def test_p11_lse_no_overflow_and_shift(orc):
    """A loud signal (ln L ~ 1e4) does not overflow, and ln L_tmarg equals the
    log of the bin mean; adding C to every ln w shifts ln Z by C and leaves
    n_eff, n_ESS unchanged."""
    p = copy.copy(S.plain_fp64_problem())
    p.Q = p.Q * 50.0
    p.U = p.U * 50.0
    p.V = p.V * 50.0
    th = S.prior_samples(50, 19)
    ll, bins, _ = orc.lnL(p, th, want_bins=True)
    assert np.all(np.isfinite(ll)) and np.max(ll) > 3000
    mx = bins.max(1)
    ref = mx + np.log(np.mean(np.exp(bins - mx[:, None]), 1))
    assert np.max(np.abs(ll - ref)) < 1e-9 * np.max(np.abs(ll))
    lnw = np.random.default_rng(2).normal(0, 3, 1000)
    r0, r1 = orc.reduce(lnw), orc.reduce(lnw + 1234.5)
    assert abs(r1["lnZ"] - r0["lnZ"] - 1234.5) < 1e-9
    assert abs(r1["n_eff"] - r0["n_eff"]) < 1e-9 * r0["n_eff"]
    assert abs(r1["n_ess"] - r0["n_ess"]) < 1e-9 * r0["n_ess"]


def test_reduce_definitions_brute_force(orc):
    """ln Z, n_eff, n_ESS, sigma against their definitions in long double via
    math.fsum on small samples (no max-subtraction)."""
    lnw = np.random.default_rng(3).normal(0, 1, 500)
    r = orc.reduce(lnw)
    w = np.exp(lnw)
    s1, s2 = math.fsum(w), math.fsum(w * w)
    assert abs(r["lnZ"] - math.log(s1 / 500)) < 1e-12
    assert abs(r["n_eff"] - s1 / w.max()) < 1e-10 * r["n_eff"]
    assert abs(r["n_ess"] - s1 * s1 / s2) < 1e-10 * r["n_ess"]
    assert abs(r["sigma_lnZ"] - math.sqrt(s2 / s1 ** 2 - 1 / 500)) < 1e-10


def test_window_violation_is_an_error(orc):
    p = copy.copy(S.plain_fp64_problem())
    p.q_t0 = np.array([-0.06, -0.1])
    with pytest.raises(ValueError):
        orc.lnL(p, S.prior_samples(200, 1))


# ---- P9 / P10 / P13 / P14: sampler and estimator ---------------------------------------

def load_philox_kat():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = []
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_p14_philox_known_answers(orc):
    """Philox4x32-10 known-answer values published with the generator."""
    kat = load_philox_kat()
    assert len(kat) == 3
    for ctr, key, out in kat:
        assert list(orc.philox4x32_10(ctr, key)) == out


def test_p13_uniform_histogram_draws_the_prior(orc):
    """Iteration 0 (uniform masses) draws the isotropic prior exactly, with
    ln p - ln p_s = 0; Kolmogorov-Smirnov against each 1-D prior CDF."""
    from scipy import stats
    sm = orc.Sampler(n_bins=32, seed=77)
    th, lr, bins = sm.draw(40000)
    assert np.all(lr == 0)
    cdfs = [lambda a: a / (2 * np.pi), lambda d: (np.sin(d) + 1) / 2, lambda s: s / np.pi,
            lambda f: f / (2 * np.pi), lambda i: (1 - np.cos(i)) / 2,
            lambda D: (D ** 3 - 100.0 ** 3) / (1000.0 ** 3 - 100.0 ** 3)]
    for d in range(6):
        assert stats.kstest(th[:, d], cdfs[d]).pvalue > 1e-3
    assert np.all(bins >= 0) and np.all(bins < 32)


def test_p13_histogram_density_and_weights(orc):
    """A non-uniform histogram: bin occupancy follows its masses (chi-square)
    and ln p - ln p_s = -sum_d ln(B P_d[b_d])."""
    from scipy import stats
    sm = orc.Sampler(n_bins=16, seed=78)
    rng = np.random.default_rng(0)
    sm.P = rng.uniform(0.2, 2.0, (6, 16))
    sm.P /= sm.P.sum(1, keepdims=True)
    n = 60000
    th, lr, bins = sm.draw(n)
    for d in range(6):
        cnt = np.bincount(bins[:, d], minlength=16)
        assert stats.chisquare(cnt, n * sm.P[d]).pvalue > 1e-4
    exp = -np.sum(np.log(16 * sm.P[np.arange(6)[None, :], bins]), 1)
    assert np.max(np.abs(lr - exp)) < 1e-12
    # the draw's v within the chosen bin: alpha = 2 pi v must sit inside bin b
    v = th[:, 0] / (2 * np.pi)
    assert np.all(np.floor(v * 16) == bins[:, 0])


def test_p13_adapt_converges_to_binned_target(orc):
    """Adapting on an analytic Gaussian weight in one unit coordinate moves
    that dimension's P_d to (1-eps) x the target's binned mass + eps/B and
    leaves the other dimensions near uniform (MC error ~1e-3)."""
    from scipy import stats
    n = 300000
    base = orc.Sampler(n_bins=20, seed=79, floor=0.1)
    th, lr, bins = base.draw(n)
    v = np.stack([th[:, 0] / (2 * np.pi), (np.sin(th[:, 1]) + 1) / 2, th[:, 2] / np.pi, th[:, 3] / (2 * np.pi),
                  (1 - np.cos(th[:, 4])) / 2, (th[:, 5] ** 3 - 1e6) / (1e9 - 1e6)], 1)
    mu, sd = 0.37, 0.12
    edges = np.linspace(0, 1, 21)
    mass = np.diff(stats.norm.cdf(edges, mu, sd))
    mass /= mass.sum()
    target = 0.9 * mass + 0.1 / 20
    for d in range(6):
        sm = orc.Sampler(n_bins=20, seed=79, floor=0.1)
        sm.adapt(bins, -0.5 * ((v[:, d] - mu) / sd) ** 2 + lr)
        assert np.max(np.abs(sm.P[d] - target)) < 0.006
        others = np.delete(np.arange(6), d)
        assert np.max(np.abs(sm.P[others] - 0.05)) < 0.006


def test_p9_zero_signal(orc):
    """Q = U = V = 0: ln L_tmarg = 0 exactly; with p_s = p, ln Z = 0 and
    n_eff = n_ESS = N; with an adapted p_s, ln Z = ln mean(p/p_s) -> 0 within 4 sigma."""
    p = S.zero_problem(S.plain_fp64_problem())
    sm = orc.Sampler(n_bins=16, seed=80)
    res = orc.run_adapt(p, sm, 1, 5000, adapt_last=False)
    it = res["iterations"][0]
    assert np.all(res["lnL"][0] == 0.0)
    assert it["lnZ"] == 0.0 and it["n_eff"] == 5000 and it["n_ess"] == 5000
    sm.P = np.random.default_rng(1).uniform(0.3, 3, (6, 16))
    sm.P /= sm.P.sum(1, keepdims=True)
    res = orc.run_adapt(p, sm, 1, 20000)
    it = res["iterations"][0]
    assert abs(it["lnZ"]) < 4 * it["sigma_lnZ"] + 1e-12


@pytest.mark.slow
def test_p10_mc_matches_quadrature(orc):
    """Tiny problem (1 detector, modes (2,+-2), 101 bins, SNR 4): the Monte
    Carlo ln Z, before and after one adaptation, agrees with a 6-D
    Gauss-Legendre product quadrature over the unit cube of prior CDF
    coordinates within 4 sigma (plus the quadrature's own error)."""
    p = S.make_problem(("H1",), 2, 4096.0, n_t=101, snr=4.0, noise=False, seed=23)
    npts = 7
    x, w = np.polynomial.legendre.leggauss(npts)
    x, w = 0.5 * (x + 1), 0.5 * w
    grids = np.meshgrid(*([x] * 6), indexing="ij")
    v = np.stack([g.ravel() for g in grids], 1)
    wt = np.prod(np.stack(np.meshgrid(*([w] * 6), indexing="ij")), 0).ravel()
    th = np.stack([2 * np.pi * v[:, 0], np.arcsin(2 * v[:, 1] - 1), np.pi * v[:, 2], 2 * np.pi * v[:, 3],
                   np.arccos(1 - 2 * v[:, 4]), np.cbrt(1e6 + v[:, 5] * (1e9 - 1e6))], 1)
    ll = orc.lnL(p, th)
    mx = ll.max()
    lnZ_q = mx + math.log(np.sum(wt * np.exp(ll - mx)))
    sm = orc.Sampler(n_bins=16, seed=81)
    res = orc.run_adapt(p, sm, 2, 200000)
    for it in res["iterations"]:
        assert abs(it["lnZ"] - lnZ_q) < 4 * it["sigma_lnZ"] + 2e-3


# ------------------------------------------------------------------------------ fair draws

def test_fair_fixed_point_weights_and_choice_definition(orc):
    """Exact integer weights W_i = floor(exp(x_i - max) 2^S), S = 62 - ceil(log2 n),
    and the choice 'first running sum above floor(U Total / 2^53)' at the ends and
    at exact interior fractions."""
    x = np.log(np.array([1.0, 2.0, 0.0, 5.0, 2.0]))   # ln 0 = -inf: never chosen
    cum, S = orc.fix_cumulative(x)
    assert S == 62 - 3
    mx = math.log(5.0)
    w = [int(math.ldexp(math.exp(v - mx), S)) if np.isfinite(v) else 0 for v in x]
    assert w[3] == 1 << S and w[2] == 0 and abs(w[0] - (1 << S) // 5) <= 64
    assert [int(c) for c in cum] == list(np.cumsum(np.array(w, dtype=object)))
    tot = int(cum[-1])
    assert orc.fix_choose(cum, 0) == 0
    assert orc.fix_choose(cum, (1 << 53) - 1) == 4
    # at each running-sum boundary c: the smallest U whose threshold floor(U tot / 2^53)
    # reaches c chooses the next item with weight; the U just below chooses the item
    # that ends at c
    for c, before, after in ((int(cum[0]), 0, 1), (int(cum[1]), 1, 3), (int(cum[3]), 3, 4)):
        U = -(-(c << 53) // tot)
        assert (U * tot) >> 53 >= c and ((U - 1) * tot) >> 53 < c
        assert orc.fix_choose(cum, U) == after
        assert orc.fix_choose(cum, U - 1) == before
    with pytest.raises(ValueError):
        orc.fix_cumulative(np.full(3, -np.inf))


def test_fair_draw_words_are_philox(orc):
    """The draw integers are Philox4x32-10 words under the reserved counter word."""
    seed, d = 0x0123456789ABCDEF, 77
    r = orc.philox4x32_10([d, 0, 0xFFFFFFFF, 0], [seed & 0xFFFFFFFF, seed >> 32])
    U = orc.fair_words(seed, d)
    assert U[0] == (int(r[0]) >> 5 << 26) | (int(r[1]) >> 6)
    assert U[1] == (int(r[2]) >> 5 << 26) | (int(r[3]) >> 6)


def test_fair_draw_frequencies_are_multinomial(orc):
    """200k draws from five weighted items: chi-square against the exact
    probabilities w_i / sum w (the p-value floor is fixed for the fixed seed)."""
    scipy_stats = pytest.importorskip("scipy.stats")
    w = np.array([0.1, 3.0, 0.0, 1.5, 0.4])
    lnw = np.log(w)
    n_draws = 200000
    idx = np.empty(n_draws, np.int64)
    cum, _ = orc.fix_cumulative(lnw)
    for d in range(n_draws):
        idx[d] = orc.fix_choose(cum, orc.fair_words(5, d)[0])
    counts = np.bincount(idx, minlength=5)
    assert counts[2] == 0
    keep = w > 0
    p = scipy_stats.chisquare(counts[keep], n_draws * w[keep] / w.sum()).pvalue
    assert p > 1e-3


def test_fair_draws_brute_force_joint_distribution(orc):
    """Tiny problem: the joint frequency of (sample, time bin) over 60000 draws
    matches w_i / sum w x exp(ln L_ij) / sum_j exp(ln L_ij) computed directly."""
    scipy_stats = pytest.importorskip("scipy.stats")
    p = S.make_problem(("H1",), 2, 4096.0, n_t=5, snr=3.0, t_lo=-0.002, t_hi=0.002, seed=31)
    th = S.prior_samples(4, 9)
    ll, bins, _ = orc.lnL(p, th, want_bins=True)
    lnw = ll + np.array([0.0, -0.5, 0.3, -1.0])
    n_draws = 60000
    idx, th_d, j, t = orc.fair_draws(p, th, lnw, n_draws, seed=12)
    assert np.array_equal(th_d, th[idx])
    assert np.allclose(t, p.t_lo + j * (p.t_hi - p.t_lo) / (p.n_t - 1), rtol=0, atol=1e-15)
    pw = np.exp(lnw - lnw.max())
    pw /= pw.sum()
    pt = np.exp(bins - bins.max(1, keepdims=True))
    pt /= pt.sum(1, keepdims=True)
    expected = (pw[:, None] * pt).ravel() * n_draws
    counts = np.bincount(idx * p.n_t + j, minlength=4 * p.n_t)
    keep = expected > 5
    assert counts[~keep].sum() < 50
    pval = scipy_stats.chisquare(counts[keep], expected[keep] * counts[keep].sum() / expected[keep].sum()).pvalue
    assert pval > 1e-3


def test_fair_time_bin_follows_a_dominant_bin(orc):
    """A bin 50 above every other is always the one drawn; equal bins are drawn
    uniformly."""
    row = np.zeros(9)
    row[6] = 50.0
    cum, _ = orc.fix_cumulative(row)
    assert all(orc.fix_choose(cum, orc.fair_words(3, d)[1]) == 6 for d in range(500))
    cum, _ = orc.fix_cumulative(np.zeros(4))
    got = np.bincount([orc.fix_choose(cum, orc.fair_words(3, d)[1]) for d in range(4000)], minlength=4)
    assert np.all(np.abs(got - 1000) < 150)


# ------------------------------------------------------------------------------ adaptive volume

def _v_of_theta(th, d_min=100.0, d_max=1000.0):
    """Prior-CDF coordinates of theta (the inverse of the draw's mapping)."""
    v = np.empty_like(th)
    v[:, 0] = th[:, 0] / (2 * np.pi)
    v[:, 1] = (np.sin(th[:, 1]) + 1) / 2
    v[:, 2] = th[:, 2] / np.pi
    v[:, 3] = th[:, 3] / (2 * np.pi)
    v[:, 4] = (1 - np.cos(th[:, 4])) / 2
    v[:, 5] = (th[:, 5] ** 3 - d_min ** 3) / (d_max ** 3 - d_min ** 3)
    return v


def test_av_draws_are_uniform_in_the_active_cells(orc):
    """Draws land only in active cells, equally often in each, and their theta is the
    prior mapping of v."""
    from oracle import av as A
    a = A.AV(seed=4)
    a.level = 2
    a.cells = np.array(sorted({int(k) for k in A.cell_keys(np.random.default_rng(0).random((5, 6)), 2)}), np.uint64)
    th, v = a.draw(40000)
    keys = A.cell_keys(v, 2)
    assert set(np.unique(keys)) <= set(a.cells.tolist())
    counts = np.array([np.sum(keys == c) for c in a.cells])
    assert np.all(np.abs(counts - 40000 / a.cells.size) < 5 * np.sqrt(40000 / a.cells.size))
    assert np.allclose(_v_of_theta(th), v, atol=1e-9)


def test_av_threshold_rule_against_sorted_definition(orc):
    """The histogram threshold keeps every point of the exact sort-based rule (the
    fewest top points holding P_thr of the mass, and at least N_min* of them) and at
    most the rest of the 1/64-wide bin where that rule stops."""
    from oracle import av as A
    rng = np.random.default_rng(2)
    for p_thr, nstar in ((0.999, 1000), (0.9, 50), (0.99999, 10)):
        lnL = rng.normal(0, 4, 5000)
        m, b_thr, kept = A.threshold(lnL, p_thr, nstar)
        order = np.argsort(-lnL)
        w = np.exp(lnL[order] - m)
        frac = np.cumsum(w) / w.sum()
        k_mass = int(np.searchsorted(frac, np.floor(p_thr * 2 ** 20) / 2 ** 20 * (1 - 1e-12))) + 1
        k = max(k_mass, nstar)
        exact = np.zeros(lnL.size, bool)
        exact[order[:k]] = True
        assert np.all(kept[exact])
        last = lnL[order[k - 1]]
        assert np.all(lnL[kept] >= last - 1.0 / 64)


def test_av_uniform_target_is_exact(orc):
    """ln L = 0: every iteration keeps all points, every cell of the chosen level stays
    active, V = 1 and ln Z = 0 exactly."""
    from oracle import av as A
    res = A.run(lambda th: np.zeros(th.shape[0]), 4, 50000, seed=5)
    for r in res["iterations"]:
        assert r["V"] == 1.0 and r["reduce"]["lnZ"] == 0.0
    assert res["iterations"][-1]["level"] >= 1


def test_av_box_target_is_exact(orc):
    """L = 1 on a box that is one cell of the level-2 grid, negligible elsewhere:
    after one refinement the active region is exactly that box (one level-2 cell, or
    all its sub-cells once the grid refines further) and ln Z = ln(4^-6) exactly."""
    from oracle import av as A
    lo = np.array([1, 2, 1, 3, 0, 2]) / 4.0

    def lnL(th):
        v = _v_of_theta(th)
        inside = np.all((v >= lo) & (v < lo + 0.25), 1)
        return np.where(inside, 0.0, -200.0)

    res = A.run(lnL, 3, 200000, seed=6, n_min_star=30)   # below the ~49 points the box holds
    its = res["iterations"]
    for r in its[1:]:
        assert r["level"] >= 2 and r["n_cells"] == 64 ** (r["level"] - 2)
        assert r["V"] == 4.0 ** -6
        assert r["reduce"]["lnZ"] == pytest.approx(-6 * math.log(4.0), abs=1e-12)


def test_av_refinement_formula_and_nesting(orc):
    """n_bins = (1/dV)^(1/6) rounded down to a power of two, never coarser; refined
    cells lie inside cells that were active."""
    from oracle import av as A
    assert A.next_level(0, 1.0, 100, 10000) == int(math.floor(math.log2((1 / (0.01 / 10)) ** (1 / 6))))
    assert A.next_level(3, 1.0, 100, 10000) == 3
    assert A.next_level(0, 1e-30, 100, 100) == A.MAX_LEVEL
    mu, sig = np.array([0.3, 0.6, 0.45, 0.55, 0.4, 0.7]), 0.05

    def lnL(th):
        return -np.sum((_v_of_theta(th) - mu) ** 2, 1) / (2 * sig ** 2)

    a = A.AV(seed=7, n_min_star=200)
    for _ in range(4):
        old_level, old_cells = a.level, set(a.cells.tolist())
        a.step(lnL, 50000)
        if a.level >= old_level:
            shift = a.level - old_level
            c = a.cells.astype(np.uint64)
            parent = np.zeros_like(c)
            for d in range(6):
                coord = (c >> np.uint64(a.level * d)) & np.uint64((1 << a.level) - 1)
                parent |= (coord >> np.uint64(shift)) << np.uint64(old_level * d)
            assert set(parent.tolist()) <= old_cells


def test_av_sharp_gaussian_keeps_n_min_floor_and_converges(orc):
    """A 6-D Gaussian with sigma = 0.002 (a posterior volume ~1e-16 of the cube): in
    iteration 0 the few draws nearest the peak hold P_thr of the mass, so the P_thr rule
    alone would keep a handful of points.  N_min* is a floor (Sec. IV A: while the
    likelihood is poorly resolved the top N_min* points are kept), so the live set keeps
    N_min* points, the region shrinks steadily instead of collapsing onto those few, and
    the late iterations' ln Z meet the analytic integral within 4 sigma + 1e-3."""
    from oracle import av as A
    mu = np.array([0.3125, 0.5625, 0.4375, 0.6875, 0.1875, 0.8125]) + 0.0004
    sig = 0.002

    def lnL(th):
        return -np.sum((_v_of_theta(th) - mu) ** 2, 1) / (2 * sig ** 2)

    truth = 3 * math.log(2 * math.pi * sig ** 2)
    a = A.AV(seed=8, n_min_star=1000)
    ll0 = lnL(A.AV(seed=8).draw(100000, it=0)[0])
    # the P_thr rule alone (no floor) keeps a handful of points in iteration 0
    assert int(A.threshold(ll0, a.p_thr, 1)[2].sum()) < 10
    its = [a.step(lnL, 100000) for _ in range(16)]
    assert its[0]["n_min"] >= 1000
    assert all(r["n_min"] >= 1000 for r in its)
    assert its[-1]["level"] >= 6
    for r in its[-3:]:
        red = A.reduce(r["lnw"])
        assert abs(red["lnZ"] - truth) < 4 * red["sigma_lnZ"] + 1e-3, (red, truth)
    assert A.reduce(its[-1]["lnw"])["n_eff"] > 20


def test_av_gaussian_target(orc):
    """A 6-D Gaussian well inside one level-3 cell on every axis (sigma = 0.01):
    each refined iteration's ln Z is within 4 sigma + 1e-3 of the analytic integral."""
    from oracle import av as A
    mu, sig = np.array([0.3125, 0.5625, 0.4375, 0.6875, 0.1875, 0.8125]), 0.01

    def lnL(th):
        return -np.sum((_v_of_theta(th) - mu) ** 2, 1) / (2 * sig ** 2)

    truth = 3 * math.log(2 * math.pi * sig ** 2)
    res = A.run(lnL, 6, 100000, seed=8, n_min_star=300)
    late = res["iterations"][3:]
    assert all(r["level"] >= 2 for r in late)
    for r in late:
        assert abs(r["reduce"]["lnZ"] - truth) < 4 * r["reduce"]["sigma_lnZ"] + 1e-3, (r["reduce"], truth)


# ------------------------------------------------------------------------------ Q, U, V from waveforms

def test_overlaps_identities(orc):
    """Q, U, V from the frequency-domain inputs: U Hermitian, V symmetric, and for
    noise-free data of mode amplitudes a arriving at t_arr, Q(t_arr) = 1/2 (U a +
    conj(V) conj(a)) exactly (the data's transform is 1/2 sum a h + conj(a) conj(h(-f)))."""
    from oracle import precompute as PC
    p = S.make_problem(("H1", "V1"), 5, 4096.0, snr=20.0, noise=False, seed=61)
    wf, data = p.meta["waveforms"], p.meta["data"]
    Q, U, V = PC.overlaps(wf.freqs, wf.h, data, wf.w, p.q_t0, p.fs, p.n_q)
    assert np.allclose(U, np.conj(np.transpose(U, (0, 2, 1))), atol=1e-12)
    assert np.allclose(V, np.transpose(V, (0, 2, 1)), atol=1e-12)
    a = p.meta["a_true"]
    for k in range(2):
        t_arr = p.meta["t_true"] + p.meta["dt_true"][k]
        t = np.array([t_arr])
        phase = np.exp(2j * np.pi * np.outer(t, wf.freqs))
        q_arr = 2.0 * (phase @ (wf.w[k] * np.conj(wf.h) * data[k]).T)[0]
        assert np.allclose(q_arr, 0.5 * (U[k] @ a[k] + np.conj(V[k]) @ np.conj(a[k])), rtol=1e-11, atol=1e-11)
    # the decomposed likelihood built from these overlaps is <h|d> - 1/2 <h|h>
    rng = np.random.default_rng(3)
    c = rng.normal(size=(2, 5)) + 1j * rng.normal(size=(2, 5))
    q_at = [Q[k, :, 0] for k in range(2)]
    lin = sum(np.real(np.vdot(c[k], q_at[k])) for k in range(2))
    quad = 0.25 * sum(np.real(np.vdot(c[k], U[k] @ c[k])) + np.real(c[k] @ V[k] @ c[k]) for k in range(2))
    t0 = np.array(p.q_t0)
    direct = 0.0
    for k in range(2):
        hk = wf.strain(c[k], t0[k])   # template arriving at Q sample 0
        direct += np.real(wf.inner(k, hk, data[k])) - 0.5 * np.real(wf.inner(k, hk, hk))
    assert lin - quad == pytest.approx(direct, rel=1e-10, abs=1e-9)


def test_overlaps_single_line_closed_form(orc):
    """One frequency line (and its mirror) in the data and one mode: Q is the closed-form
    sinusoid 2 w conj(h) d exp(2 pi i f t) summed over the two lines."""
    from oracle import precompute as PC
    f = np.array([-10.0, -6.0, 6.0, 10.0])
    h = np.array([[0.0, 1.0 + 0.5j, 0.2 - 0.1j, 0.0]])
    d = np.array([[0.0, 0.3 - 0.7j, 0.3 + 0.7j, 0.0]])
    w = np.array([[1.0, 1.5, 1.5, 1.0]])
    Q, U, V = PC.overlaps(f, h, d, w, np.array([-0.1]), 100.0, 50)
    t = -0.1 + np.arange(50) / 100.0
    exp = 2 * 1.5 * (np.conj(h[0, 1]) * d[0, 1] * np.exp(2j * np.pi * -6.0 * t)
                     + np.conj(h[0, 2]) * d[0, 2] * np.exp(2j * np.pi * 6.0 * t))
    assert np.allclose(Q[0, 0], exp, atol=1e-13)
    assert U[0, 0, 0] == pytest.approx(2 * 1.5 * (abs(h[0, 1]) ** 2 + abs(h[0, 2]) ** 2))
    assert V[0, 0, 0] == pytest.approx(2 * 1.5 * 2 * h[0, 1] * h[0, 2])


# ------------------------------------------------------------------------------ distance marginalisation

DREF, DMIN, DMAX = 400.0, 100.0, 1000.0


def test_dist_marg_zero_signal_is_the_prior_normalisation(orc):
    assert abs(orc.ln_dist_marg(0.0, 0.0, DREF, DMIN, DMAX)) < 1e-13
    assert abs(orc.ln_dist_marg(0.0, 0.0, 250.0, 50.0, 2000.0)) < 1e-13


@pytest.mark.parametrize("a,b", [(3.0, 1.0), (40.0, 12.0), (-5.0, 2.0), (150.0, 30.0), (900.0, 400.0),
                                 (0.5, 0.0), (-30.0, 0.0)])
def test_dist_marg_against_library_quadrature_in_distance(orc, a, b):
    """The integral over D of p(D) exp(a x - b x^2), x = D_ref/D, by scipy's adaptive
    quadrature in D (with the peak as a break point)."""
    integrate = pytest.importorskip("scipy.integrate")
    norm = 3.0 / (DMAX ** 3 - DMIN ** 3)
    x = lambda D: DREF / D
    xm = a / (2 * b) if b > 0 else (DREF / DMIN if a > 0 else DREF / DMAX)
    xm = min(max(xm, DREF / DMAX), DREF / DMIN)
    shift = a * xm - b * xm * xm
    f = lambda D: norm * D * D * math.exp(a * x(D) - b * x(D) ** 2 - shift)
    pts = [DREF / xm] if DMIN < DREF / xm < DMAX else None
    val, err = integrate.quad(f, DMIN, DMAX, points=pts, epsabs=0, epsrel=1e-13, limit=500)
    assert orc.ln_dist_marg(a, b, DREF, DMIN, DMAX) == pytest.approx(shift + math.log(val), abs=1e-10)


def test_dist_marg_laplace_limit(orc):
    """A sharp peak well inside the distance range: ln I tends to the Laplace value
    ln C + a^2/4b - 4 ln x* + ln sqrt(pi/b), with an error falling like 1/(b x*^2)."""
    lnC = math.log(3 * DREF ** 3 / (DMAX ** 3 - DMIN ** 3))
    xs = 1.3
    errs = []
    for bx2 in (1e3, 4e3, 1.6e4):
        b = bx2 / xs ** 2
        a = 2 * b * xs
        lap = lnC + a * a / (4 * b) - 4 * math.log(xs) + 0.5 * math.log(math.pi / b)
        errs.append(abs(orc.ln_dist_marg(a, b, DREF, DMIN, DMAX) - lap))
    assert errs[-1] < 1e-3
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3


def test_dist_marg_likelihood_brute_force_over_a_distance_grid(orc):
    """Per-bin distance-marginal ln L of the whole chain against the average over a
    Gauss-Legendre grid in D of the ordinary per-bin likelihood at each D."""
    p = S.make_problem(("H1", "L1"), 4, 4096.0, n_t=41, t_lo=-0.005, t_hi=0.005, snr=6.0, seed=81)
    th = S.prior_samples(6, 4)
    Pm = orc.Problem(p, dist_marg=True)
    _, mb, _ = orc.lnL(Pm, th, want_bins=True)
    xg, wg = np.polynomial.legendre.leggauss(48)
    edges = np.linspace(p.d_min, p.d_max, 41)
    Ds = ((edges[:-1, None] + edges[1:, None]) / 2 + (edges[1:, None] - edges[:-1, None]) / 2 * xg).ravel()
    Ws = ((edges[1:, None] - edges[:-1, None]) / 2 * wg).ravel() * 3 * Ds ** 2 / (p.d_max ** 3 - p.d_min ** 3)
    for i in range(th.shape[0]):
        rows = np.repeat(th[i:i + 1], Ds.size, 0)
        rows[:, 5] = Ds
        _, bins, _ = orc.lnL(p, rows, want_bins=True)      # [nD][n_t]
        m = bins.max(0)
        brute = m + np.log(np.sum(Ws[:, None] * np.exp(bins - m), 0))
        assert np.allclose(mb[i], brute, atol=1e-8, rtol=1e-10), np.max(np.abs(mb[i] - brute))


def test_dist_marg_sampler_drops_the_distance_weight(orc):
    rng = np.random.default_rng(5)
    P = rng.uniform(0.2, 3.0, (6, 16))
    P /= P.sum(1, keepdims=True)
    full, marg = orc.Sampler(n_bins=16, seed=3), orc.Sampler(n_bins=16, seed=3, dist_marg=True)
    full.P, marg.P = P.copy(), P.copy()
    thf, lrf, bf = full.draw(500)
    thm, lrm, bm = marg.draw(500)
    assert np.array_equal(thf, thm) and np.array_equal(bf, bm)
    assert np.allclose(lrf - lrm, -np.log(16 * P[5, bf[:, 5]]), atol=1e-12)
    marg.adapt(bm, rng.normal(0, 3, 500))
    assert np.array_equal(marg.P[5], P[5]) and not np.allclose(marg.P[:5], P[:5])
