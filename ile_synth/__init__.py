"""Seeded synthetic inputs for the extrinsic-marginalised likelihood (ILE).

This module is shared by the tests, the oracle-driven checks and the
benchmark.  It builds *inputs only*: detector geometry, frequency-domain mode
waveforms, the overlaps Q, U, V that the likelihood consumes, and extrinsic
sample sets.  It contains none of the likelihood arithmetic (no antenna
pattern, no spin-weighted harmonic, no decomposed log-likelihood, no
time marginalisation, no Monte Carlo reduction, no sampler).

Everything is computed from the paper's definitions of the inner products
(arXiv:2505.11655, Sec. II A, Eq. (QUV)): with a discrete two-sided frequency
grid f in {+-f_1..+-f_F} and inverse-PSD weights w_k(f),

    <a|b>_k        = 2 sum_f w_k(f) conj(a~(f)) b~(f)
    Q_k,lm(t)      = 2 sum_f w_k(f) exp(2 pi i f t) conj(h~_lm(f)) d~_k(f)
    U_k,lm,l'm'    = <h_lm | h_l'm'>_k
    V_k,lm,l'm'    = <conj(h_lm) | h_l'm'>_k = 2 sum_f w_k(f) h~_lm(-f) h~_l'm'(f)

The injected detector signal for complex mode coefficients a_k,lm is the real
strain h_k(t) = Re sum_lm a_k,lm h_lm(t - t_arr,k), whose transform is
1/2 sum_lm [a h~_lm(f) + conj(a) conj(h~_lm(-f))] exp(-2 pi i f t_arr,k).
Its optimal SNR is rho^2 = sum_k <h_k|h_k>_k, taken directly from the
waveforms.  Real noise n_k has n~(f) ~ CN(0, 1/(2 w_k(f))) for f > 0 and
n~(-f) = conj(n~(f)), so that Var<h|n> = <h|h>.

Default injections draw the per-detector response factor and the per-mode
angular factor as random complex numbers of realistic size (|F| in [0.3, 1],
|Y| ~ 0.3) rather than evaluating them at a "true" sky position; callers that
need a physically realisable injection pass ``a0`` (the product F_k Y_lm at
unit distance ratio) and ``dt_true`` themselves.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

C_SI = 299792458.0

# Mode order (l, m): the first M entries are used for an M-mode problem.
MODE_ORDER = [(2, 2), (2, -2), (2, 1), (2, -1), (3, 3), (3, -3), (2, 0), (3, 2), (3, -2),
              (4, 4), (4, -4), (3, 1), (3, -1), (4, 3), (4, -3), (3, 0), (4, 2), (4, -2),
              (4, 1), (4, -1), (4, 0)]

# Amplitude hierarchy s_lm of the synthetic mode waveforms (by |m| and l).
S_DEFAULT = {(2, 2): 1.0, (2, 1): 0.3, (3, 3): 0.3, (4, 4): 0.15}
S_Q20 = {(2, 2): 1.0, (2, 1): 0.5, (3, 3): 0.7, (3, 2): 0.35, (4, 4): 0.45, (4, 3): 0.25}

# Approximate geodetic description of the detectors (vertex latitude and
# longitude in degrees, elevation in metres, arm azimuths in degrees clockwise
# from North, arm altitudes in radians).  These are rounded published survey
# values, accurate to roughly 1e-4 degrees; they only shape the synthetic
# workload, both implementations receive the resulting tensors as inputs.
DETECTORS = {
    "H1": (46.455144, -119.407656, 142.554, 324.000, 234.000, -6.195e-4, 1.25e-5),
    "L1": (30.562894, -90.774242, -6.574, 252.2835, 162.2835, -3.121e-4, -6.107e-4),
    "V1": (43.631414, 10.504498, 51.884, 19.4326, 289.4326, 0.0, 0.0),
    # a synthetic fourth site (southern hemisphere, arms at 20 and 110 degrees), used only
    # for four-detector test problems
    "X1": (-31.0, 115.0, 0.0, 20.0, 110.0, 0.0, 0.0),
}


def detector_geometry(name: str):
    """Detector response tensor D = (u u^T - v v^T)/2 and vertex position (m).

    Earth-fixed Cartesian frame, WGS-84 ellipsoid; u, v are the arm unit
    vectors built from the local East/North/Up frame at the vertex.
    """
    lat_d, lon_d, elev, az_x, az_y, alt_x, alt_y = DETECTORS[name]
    lat, lon = math.radians(lat_d), math.radians(lon_d)
    a, f = 6378137.0, 1.0 / 298.257223563
    e2 = f * (2.0 - f)
    n = a / math.sqrt(1.0 - e2 * math.sin(lat) ** 2)
    pos = np.array([(n + elev) * math.cos(lat) * math.cos(lon),
                    (n + elev) * math.cos(lat) * math.sin(lon),
                    (n * (1.0 - e2) + elev) * math.sin(lat)])
    east = np.array([-math.sin(lon), math.cos(lon), 0.0])
    north = np.array([-math.sin(lat) * math.cos(lon), -math.sin(lat) * math.sin(lon), math.cos(lat)])
    up = np.array([math.cos(lat) * math.cos(lon), math.cos(lat) * math.sin(lon), math.sin(lat)])

    def arm(az_deg, alt):
        az = math.radians(az_deg)
        return math.cos(alt) * (math.sin(az) * east + math.cos(az) * north) + math.sin(alt) * up

    u, v = arm(az_x, alt_x), arm(az_y, alt_y)
    tensor = 0.5 * (np.outer(u, u) - np.outer(v, v))
    return tensor, pos


def mode_amplitude(l: int, m: int, table: dict) -> float:
    return table.get((l, abs(m)), 0.1 if table is S_Q20 else 0.05)


@dataclass
class Problem:
    """Everything the likelihood needs for one intrinsic point (host arrays)."""
    det_names: list
    det_tensor: np.ndarray      # [K][3][3] float64
    det_pos: np.ndarray         # [K][3] float64 (m)
    gmst: float
    lm: np.ndarray              # [M][2] int32
    fs: float
    n_q: int
    q_t0: np.ndarray            # [K] float64 (s, relative to the reference epoch)
    Q: np.ndarray               # [K][M][n_q] complex128
    U: np.ndarray               # [K][M][M] complex128
    V: np.ndarray               # [K][M][M] complex128
    t_lo: float
    t_hi: float
    n_t: int
    d_ref: float
    d_min: float = 100.0
    d_max: float = 1000.0
    quad_norm: int = 0          # 0: quarter (paper), 1: half
    meta: dict = field(default_factory=dict)

    @property
    def n_det(self):
        return int(self.det_tensor.shape[0])

    @property
    def n_modes(self):
        return int(self.lm.shape[0])


class Waveforms:
    """Random frequency-domain mode waveforms h~_lm(f) and per-detector weights."""

    def __init__(self, lm, n_det, rng, n_freq=128, df=2.0, hierarchy=S_DEFAULT, minor=0.1):
        self.lm = [tuple(x) for x in lm]
        self.fpos = df * np.arange(1, n_freq + 1)
        # two-sided grid, negative frequencies first, mirror-symmetric
        self.freqs = np.concatenate([-self.fpos[::-1], self.fpos])
        nf = self.freqs.size
        idx = {x: i for i, x in enumerate(self.lm)}
        h = np.zeros((len(self.lm), nf), complex)

        def cn(scale, size):
            return scale * (rng.standard_normal(size) + 1j * rng.standard_normal(size)) / math.sqrt(2.0)

        neg, pos = slice(0, n_freq), slice(n_freq, nf)
        for (l, m), i in idx.items():
            if m < 0 and (l, -m) in idx:
                continue
            s = mode_amplitude(l, m, hierarchy)
            if m == 0:
                h[i, pos] = cn(s, n_freq)
                h[i, neg] = (-1) ** l * np.conj(h[i, pos][::-1])
                continue
            h[i, neg] = cn(s, n_freq)          # dominant content on one sign of f
            h[i, pos] = cn(minor * s, n_freq)
        for (l, m), i in idx.items():          # non-precessing mirror modes
            if m < 0:
                if (l, -m) in idx:
                    h[i] = (-1) ** l * np.conj(h[idx[(l, -m)]][::-1])
                else:
                    s = mode_amplitude(l, m, hierarchy)
                    h[i, pos] = cn(s, n_freq)
                    h[i, neg] = cn(minor * s, n_freq)
        self.h = h
        w_half = rng.uniform(0.5, 2.0, size=(n_det, n_freq))
        self.w = np.concatenate([w_half[:, ::-1], w_half], axis=1)   # symmetric in f

    def inner(self, k, a, b):
        """<a|b>_k for frequency-domain arrays a, b on the two-sided grid."""
        return 2.0 * np.sum(self.w[k] * np.conj(a) * b, axis=-1)

    def gram(self, k):
        h, w = self.h, self.w[k]
        U = 2.0 * (np.conj(h) * w) @ h.T
        V = 2.0 * (h[:, ::-1] * w) @ h.T
        return U, V

    def strain(self, a_k, t_arr=0.0):
        """Transform of Re sum_lm a_lm h_lm(t - t_arr)."""
        h = self.h
        hk = 0.5 * (a_k @ h + np.conj(a_k) @ np.conj(h[:, ::-1]))
        return hk * np.exp(-2j * math.pi * self.freqs * t_arr)

    def noise(self, k, rng):
        nf = self.fpos.size
        sig = np.sqrt(1.0 / (2.0 * self.w[k, nf:]))
        npos = sig * (rng.standard_normal(nf) + 1j * rng.standard_normal(nf)) / math.sqrt(2.0)
        return np.concatenate([np.conj(npos[::-1]), npos])

    def overlap_series(self, k, d_tilde, times):
        """Q_k,lm(t) at the given times for data d~ (definition, no approximation)."""
        phase = np.exp(2j * math.pi * np.outer(times, self.freqs))      # [T][F]
        kern = (self.w[k] * d_tilde)[None, :] * np.conj(self.h)          # [M][F]
        return 2.0 * (phase @ kern.T).T                                   # [M][T]


def default_modes(n_modes: int) -> np.ndarray:
    if not 1 <= n_modes <= len(MODE_ORDER):
        raise ValueError("n_modes out of range")
    return np.array(MODE_ORDER[:n_modes], dtype=np.int32)


def make_problem(det_names=("H1", "L1"), n_modes=2, fs=4096.0, window=0.2, t_lo=-0.05, t_hi=0.05,
                 n_t=401, snr=20.0, noise=True, seed=0, hierarchy=S_DEFAULT, a0=None, dt_true=None,
                 t_true=None, d_true=400.0, d_min=100.0, d_max=1000.0, gmst=None, q_t0=None,
                 n_q=None, quad_norm=0, lm=None) -> Problem:
    """Build one seeded synthetic ILE problem.

    a0[K][M]   : F_k Y_lm of the injection at unit distance ratio (drawn if None)
    dt_true[K] : arrival delay of the injection at each detector (drawn if None)
    t_true     : injected geocentric time (drawn in [-20, 20] ms if None)
    The injection amplitude is set so that sum_k <h_k|h_k> = snr^2, and D_ref
    follows from D_ref / d_true = that scale.
    """
    rng = np.random.default_rng(seed)
    K = len(det_names)
    lm = default_modes(n_modes) if lm is None else np.asarray(lm, dtype=np.int32)
    M = lm.shape[0]
    geo = [detector_geometry(n) for n in det_names]
    tens = np.array([g[0] for g in geo])
    pos = np.array([g[1] for g in geo])
    if gmst is None:
        gmst = float(rng.uniform(0.0, 2.0 * math.pi))
    wf = Waveforms(lm, K, rng, hierarchy=hierarchy)
    if a0 is None:
        fk = rng.uniform(0.3, 1.0, K) * np.exp(2j * math.pi * rng.uniform(size=K))
        ym = 0.3 * rng.uniform(0.5, 1.5, M) * np.exp(2j * math.pi * rng.uniform(size=M))
        a0 = np.outer(fk, ym)
    a0 = np.asarray(a0, complex).reshape(K, M)
    if dt_true is None:
        rmax = np.linalg.norm(pos, axis=1) / C_SI
        dt_true = rng.uniform(-1.0, 1.0, K) * rmax
    dt_true = np.asarray(dt_true, float).reshape(K)
    if t_true is None:
        t_true = float(rng.uniform(-0.02, 0.02))
    rho2_unit = sum(np.real(wf.inner(k, wf.strain(a0[k]), wf.strain(a0[k]))) for k in range(K))
    scale = snr / math.sqrt(rho2_unit) if snr > 0 else 0.0
    a_true = scale * a0
    if n_q is None:
        n_q = int(round(window * fs))
    if q_t0 is None:
        q_t0 = np.full(K, -0.5 * window)
    q_t0 = np.asarray(q_t0, float).reshape(K)
    Q = np.zeros((K, M, n_q), complex)
    U = np.zeros((K, M, M), complex)
    V = np.zeros((K, M, M), complex)
    noise_rng = np.random.default_rng(seed + 7919)
    data = np.zeros((K, wf.freqs.size), complex)
    for k in range(K):
        d = wf.strain(a_true[k], t_true + dt_true[k])
        if noise:
            d = d + wf.noise(k, noise_rng)
        data[k] = d
        times = q_t0[k] + np.arange(n_q) / fs
        Q[k] = wf.overlap_series(k, d, times)
        U[k], V[k] = wf.gram(k)
    d_ref = scale * d_true if scale > 0 else d_true
    meta = dict(seed=seed, snr=snr, a_true=a_true, dt_true=dt_true, t_true=t_true, d_true=d_true,
                scale=scale, noise=noise, waveforms=wf, data=data)
    return Problem(list(det_names), tens, pos, float(gmst), lm, float(fs), int(n_q), q_t0, Q, U, V,
                   float(t_lo), float(t_hi), int(n_t), float(d_ref), float(d_min), float(d_max),
                   int(quad_norm), meta)


def zero_problem(base: Problem) -> Problem:
    """Same geometry with Q = U = V = 0 (no signal, no noise)."""
    p = Problem(**{k: getattr(base, k) for k in base.__dataclass_fields__})
    p.Q = np.zeros_like(base.Q)
    p.U = np.zeros_like(base.U)
    p.V = np.zeros_like(base.V)
    p.meta = dict(base.meta)
    return p


def prior_samples(n: int, seed: int, d_min=100.0, d_max=1000.0) -> np.ndarray:
    """Extrinsic samples [n][6] = (alpha, delta, psi, phi, iota, D) from the
    isotropic prior: uniform alpha, psi, phi; uniform sin(delta) and cos(iota);
    D^3 uniform on [d_min^3, d_max^3]."""
    rng = np.random.default_rng(seed)
    th = np.empty((n, 6))
    th[:, 0] = rng.uniform(0.0, 2.0 * math.pi, n)
    th[:, 1] = np.arcsin(rng.uniform(-1.0, 1.0, n))
    th[:, 2] = rng.uniform(0.0, math.pi, n)
    th[:, 3] = rng.uniform(0.0, 2.0 * math.pi, n)
    th[:, 4] = np.arccos(rng.uniform(-1.0, 1.0, n))
    th[:, 5] = np.cbrt(rng.uniform(d_min ** 3, d_max ** 3, n))
    return th


# ---- the five benchmark workloads --------------------------------------------------------

BASE_SEED = 2505116550


def config_seed(config: int, point: int = 0) -> int:
    return BASE_SEED + 1000 * config + point


def plain_fp64_problem(point: int = 0) -> Problem:
    """Two detectors (H1, L1), modes (2,+-2), 4096 Hz over 0.2 s (819 samples),
    401 bins on [-50, 50] ms, SNR 20 with noise."""
    return make_problem(("H1", "L1"), 2, 4096.0, n_t=401, snr=20.0, seed=config_seed(1, point))


def single_large_problem(point: int = 0) -> Problem:
    """Three detectors, all 21 modes with 2 <= l <= 4, 16384 Hz over 0.2 s
    (3277 samples), 1001 bins on [-50, 50] ms, SNR 20 with noise."""
    return make_problem(("H1", "L1", "V1"), 21, 16384.0, n_t=1001, snr=20.0, seed=config_seed(2, point))


def high_snr_problem(snr=150.0, point: int = 0, a0=None, dt_true=None) -> Problem:
    """Three detectors, 21 modes with a q=20-like hierarchy, 16384 Hz, 1001 bins."""
    return make_problem(("H1", "L1", "V1"), 21, 16384.0, n_t=1001, snr=snr, seed=config_seed(4, point),
                        hierarchy=S_Q20, a0=a0, dt_true=dt_true)


def batched_problem_spec(point: int):
    """Per-point sizes of the batched uneven workload (512 points)."""
    rng = np.random.default_rng(config_seed(3, point))
    K = int(rng.integers(1, 4))
    M = int(rng.integers(2, 22))
    n = int(round(10 ** rng.uniform(4, 6)))
    fs = 4096.0 if M <= 4 else float(rng.choice([4096.0, 16384.0]))
    n_t = int(rng.choice([401, 1001]))
    snr = float(rng.uniform(8, 50))
    dets = ("H1", "L1", "V1")[:K]
    return dict(det_names=dets, n_modes=M, fs=fs, n_t=n_t, snr=snr, n_samples=n,
                seed=config_seed(3, point))


def batched_problem(point: int) -> tuple:
    spec = batched_problem_spec(point)
    n = spec.pop("n_samples")
    return make_problem(spec["det_names"], spec["n_modes"], spec["fs"], n_t=spec["n_t"], snr=spec["snr"],
                        seed=spec["seed"]), n
