"""FP64 CPU oracle for the extrinsic-marginalised likelihood (ILE) of arXiv:2505.11655.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  The product library
never loads it; the two implementations share no code, only the seeded input
generator in ``ile_synth`` (which holds none of the method's arithmetic).

The arithmetic lives in ``ile_oracle.c`` (plain C, double precision, one
sample at a time, OpenMP over independent samples).  This module loads it with
ctypes and composes the steps in the paper's order:

    draw (Sec. II B) -> ln L per bin (Eq. def:lnL:Decomposed) ->
    time marginal (App. timing) -> ln w = ln L + ln p - ln p_s ->
    ln Z, n_eff, n_ESS (Eqs. lnL:MonteCarlo, neff; Sec. IV A) -> adapt (Sec. II B)

Parity pins for every function are in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ile_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libile_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, -O3, no fast-math, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c11", "-O3", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(C.Structure):
    _fields_ = [
        ("n_det", C.c_int32), ("det_tensor", C.c_void_p), ("det_pos", C.c_void_p), ("gmst", C.c_double),
        ("n_modes", C.c_int32), ("lm", C.c_void_p), ("fs", C.c_double), ("n_q", C.c_int32),
        ("q_t0", C.c_void_p), ("Q", C.c_void_p), ("U", C.c_void_p), ("V", C.c_void_p),
        ("t_lo", C.c_double), ("t_hi", C.c_double), ("n_t", C.c_int32),
        ("d_ref", C.c_double), ("d_min", C.c_double), ("d_max", C.c_double), ("kappa", C.c_double),
        ("dist_marg", C.c_int32),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            P = C.POINTER(_Problem)
            vp, i64, dbl = C.c_void_p, C.c_int64, C.c_double
            L.orc_lnL_batch.argtypes = [P, vp, i64, vp, vp, vp]
            L.orc_lnL_batch.restype = i64
            L.orc_coeffs_batch.argtypes = [P, vp, i64, vp, vp, vp, vp]
            L.orc_coeffs_batch.restype = None
            L.orc_reduce.argtypes = [vp, i64, vp]
            L.orc_reduce.restype = None
            L.orc_philox4x32_10.argtypes = [vp, vp, vp]
            L.orc_philox4x32_10.restype = None
            L.orc_uniforms.argtypes = [C.c_uint64, C.c_uint32, i64, vp]
            L.orc_uniforms.restype = None
            L.orc_draw.argtypes = [vp, C.c_int, C.c_uint64, C.c_uint32, i64, i64, dbl, dbl, C.c_int, vp, vp, vp, vp]
            L.orc_portfolio_members.argtypes = [C.c_uint64, C.c_uint32, i64, dbl, dbl, vp]
            L.orc_portfolio_members.restype = None
            L.orc_ndtri.argtypes = [dbl]
            L.orc_ndtri.restype = dbl
            L.orc_gmm_draw.argtypes = [vp, vp, vp, C.c_int, C.c_uint64, C.c_uint32, i64, dbl, dbl, vp, vp, vp]
            L.orc_gmm_draw.restype = None
            L.orc_draw.restype = None
            L.orc_adapt.argtypes = [vp, C.c_int, vp, vp, i64, dbl, dbl, C.c_int]
            L.orc_adapt.restype = None
            L.orc_wigner_d.argtypes = [C.c_int, C.c_int, dbl]
            L.orc_wigner_d.restype = dbl
            L.orc_antenna.argtypes = [vp, dbl, dbl, dbl, dbl, vp, vp]
            L.orc_antenna.restype = None
            L.orc_delay.argtypes = [vp, dbl, dbl, dbl]
            L.orc_delay.restype = dbl
            L.orc_av_draw.argtypes = [vp, i64, C.c_int, C.c_uint64, C.c_uint32, i64, i64, dbl, dbl, vp, vp]
            L.orc_av_draw.restype = None
            L.orc_fair_words.argtypes = [C.c_uint64, i64, vp]
            L.orc_fair_words.restype = None
            L.orc_fix_cumulative.argtypes = [vp, i64, vp]
            L.orc_fix_cumulative.restype = C.c_int
            L.orc_fix_choose.argtypes = [vp, i64, C.c_uint64]
            L.orc_fix_choose.restype = i64
            L.orc_fair_draws.argtypes = [vp, i64, C.c_uint64, i64, vp, vp]
            L.orc_fair_draws.restype = C.c_int
            L.orc_fair_time_bin.argtypes = [vp, i64, C.c_uint64]
            L.orc_fair_time_bin.restype = i64
            L.orc_num_threads.argtypes = []
            L.orc_num_threads.restype = C.c_int
            L.orc_set_gauss_legendre16.argtypes = [vp, vp]
            L.orc_set_gauss_legendre16.restype = None
            L.orc_ln_dist_marg.argtypes = [dbl, dbl, dbl, dbl, dbl]
            L.orc_ln_dist_marg.restype = dbl
            t, w = np.polynomial.legendre.leggauss(16)
            t, w = np.ascontiguousarray(t), np.ascontiguousarray(w)
            L.orc_set_gauss_legendre16(t.ctypes.data_as(C.c_void_p), w.ctypes.data_as(C.c_void_p))
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


KAPPA = {0: 0.25, 1: 0.5}


class Problem:
    """Holds contiguous copies of a problem's arrays and the C struct pointing at them."""

    def __init__(self, prob, dist_marg=False):
        self.src = prob
        self.dist_marg = bool(dist_marg)
        self.det_tensor = np.ascontiguousarray(prob.det_tensor, dtype=np.float64)
        self.det_pos = np.ascontiguousarray(prob.det_pos, dtype=np.float64)
        self.lm = np.ascontiguousarray(prob.lm, dtype=np.int32)
        self.q_t0 = np.ascontiguousarray(prob.q_t0, dtype=np.float64)
        self.Q = np.ascontiguousarray(prob.Q, dtype=np.complex128)
        self.U = np.ascontiguousarray(prob.U, dtype=np.complex128)
        self.V = np.ascontiguousarray(prob.V, dtype=np.complex128)
        self.n_det = self.det_tensor.shape[0]
        self.n_modes = self.lm.shape[0]
        self.n_t = int(prob.n_t)
        self.d_min, self.d_max = float(prob.d_min), float(prob.d_max)
        self.s = _Problem(self.n_det, _p(self.det_tensor), _p(self.det_pos), float(prob.gmst), self.n_modes,
                          _p(self.lm), float(prob.fs), int(prob.n_q), _p(self.q_t0), _p(self.Q), _p(self.U),
                          _p(self.V), float(prob.t_lo), float(prob.t_hi), int(prob.n_t), float(prob.d_ref),
                          float(prob.d_min), float(prob.d_max), KAPPA[int(prob.quad_norm)], int(self.dist_marg))


def _as_problem(p):
    return p if isinstance(p, Problem) else Problem(p)


def lnL(prob, theta, want_bins=False):
    """ln L_tmarg [n] (and ln L per bin [n][n_t], quad [n]) for samples theta [n][6].

    Raises ValueError if any sample's interpolation nodes leave the Q window."""
    P = _as_problem(prob)
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1, 6)
    n = th.shape[0]
    out = np.empty(n)
    quad = np.empty(n)
    bins = np.empty((n, P.n_t)) if want_bins else None
    bad = lib().orc_lnL_batch(C.byref(P.s), _p(th), n, _p(bins), _p(out), _p(quad))
    if bad:
        raise ValueError(f"{bad} samples fall outside the Q window")
    return (out, bins, quad) if want_bins else out


def coeffs(prob, theta):
    """Per-sample F [n][K], Y [n][M], c [n][K][M] (complex) and dt [n][K]."""
    P = _as_problem(prob)
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1, 6)
    n = th.shape[0]
    F = np.empty((n, P.n_det), np.complex128)
    Y = np.empty((n, P.n_modes), np.complex128)
    c = np.empty((n, P.n_det, P.n_modes), np.complex128)
    dt = np.empty((n, P.n_det))
    lib().orc_coeffs_batch(C.byref(P.s), _p(th), n, _p(F), _p(Y), _p(c), _p(dt))
    return F, Y, c, dt


def reduce(lnw):
    """dict(lnZ, sigma_lnZ, n_eff, n_ess, lnw_max) of log-weights lnw."""
    a = np.ascontiguousarray(lnw, dtype=np.float64)
    out = np.empty(5)
    lib().orc_reduce(_p(a), a.size, _p(out))
    return dict(lnZ=out[0], sigma_lnZ=out[1], n_eff=out[2], n_ess=out[3], lnw_max=out[4])


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def uniforms(seed, it, i):
    out = np.empty(6)
    lib().orc_uniforms(seed, it, i, _p(out))
    return out


def wigner_d(l, m, iota):
    return lib().orc_wigner_d(l, m, iota)


def sYlm(l, m, theta, varphi):
    return np.sqrt((2 * l + 1) / (4 * np.pi)) * wigner_d(l, m, theta) * np.exp(1j * m * varphi)


def antenna(tensor, alpha, delta, psi, gmst):
    D = np.ascontiguousarray(tensor, dtype=np.float64)
    fp, fx = C.c_double(), C.c_double()
    lib().orc_antenna(_p(D), alpha, delta, psi, gmst, C.byref(fp), C.byref(fx))
    return fp.value, fx.value


def delay(pos, alpha, delta, gmst):
    x = np.ascontiguousarray(pos, dtype=np.float64)
    return lib().orc_delay(_p(x), alpha, delta, gmst)


class Sampler:
    """Product-form adaptive histogram sampling prior: masses P[6][B].  With dist_marg
    the distance coordinate is marginalised: it carries no sampling weight and its masses
    stay as they are."""

    def __init__(self, n_bins=64, seed=1, floor=0.1, temper=1.0, d_min=100.0, d_max=1000.0, dist_marg=False):
        self.B = int(n_bins)
        self.P = np.full((6, self.B), 1.0 / self.B)
        self.seed = int(seed)
        self.floor = float(floor)
        self.temper = float(temper)
        self.d_min, self.d_max = float(d_min), float(d_max)
        self.dist_marg = bool(dist_marg)
        self.iteration = 0

    def draw(self, n, it=None, i0=0, want_v=False):
        it = self.iteration if it is None else it
        th = np.empty((n, 6))
        lr = np.empty(n)
        bins = np.empty((n, 6), np.int32)
        v = np.empty((n, 6)) if want_v else None
        Pc = np.ascontiguousarray(self.P)
        lib().orc_draw(_p(Pc), self.B, self.seed, it, i0, n, self.d_min, self.d_max, int(self.dist_marg), _p(th),
                       _p(lr), _p(bins), _p(v) if want_v else None)
        return (th, lr, bins, v) if want_v else (th, lr, bins)

    def ln_density(self, v):
        """ln p_s at points v [n][6] of the unit cube (bins floor(v B)), and the bins."""
        b = np.minimum(np.floor(np.asarray(v) * self.B), self.B - 1).astype(np.int32)
        tot = np.cumsum(self.P, axis=1)[:, -1]   # the running sum, as in the draws
        lnd = np.zeros(len(b))
        for d in range(6):
            if not (self.dist_marg and d == 5):
                lnd += np.log(self.B * self.P[d, b[:, d]] / tot[d])
        return lnd, b

    def adapt(self, bins, lnw):
        Pc = np.ascontiguousarray(self.P)
        b = np.ascontiguousarray(bins, dtype=np.int32)
        w = np.ascontiguousarray(lnw, dtype=np.float64)
        lib().orc_adapt(_p(Pc), self.B, _p(b), _p(w), w.size, self.floor, self.temper, int(self.dist_marg))
        self.P = Pc


def run_adapt(prob, sampler: Sampler, n_iter: int, n_per_iter: int, adapt_last=True):
    """The adaptive ILE loop: per iteration draw -> ln L -> ln w -> reduce -> adapt.

    Returns dict(iterations=[per-iteration reduce dicts], pooled=reduce of all
    iterations' ln w, lnw=[per-iteration arrays], theta=[...], lnL=[...])."""
    P = _as_problem(prob)
    its, lnws, thetas, lnLs = [], [], [], []
    for g in range(n_iter):
        th, lr, bins = sampler.draw(n_per_iter)
        ll = lnL(P, th)
        lnw = ll + lr
        its.append(reduce(lnw))
        lnws.append(lnw)
        thetas.append(th)
        lnLs.append(ll)
        if adapt_last or g + 1 < n_iter:
            sampler.adapt(bins, lnw)
        sampler.iteration += 1
    pooled = reduce(np.concatenate(lnws))
    pooled["lnL_max"] = float(max(np.max(x) for x in lnLs))
    return dict(iterations=its, pooled=pooled, lnw=lnws, theta=thetas, lnL=lnLs)


def fair_words(seed, d):
    """53-bit integers (sample choice, time choice) of fair draw d."""
    out = np.empty(2, np.uint64)
    lib().orc_fair_words(int(seed), int(d), _p(out))
    return int(out[0]), int(out[1])


def fix_cumulative(x):
    """Running sums of the exact fixed-point weights of log-weights x, and the shift S."""
    a = np.ascontiguousarray(x, dtype=np.float64)
    cum = np.empty(max(1, a.size), np.uint64)
    S = lib().orc_fix_cumulative(_p(a), a.size, _p(cum))
    if S < 0:
        raise ValueError("no finite log-weight")
    return cum[:a.size], S


def fix_choose(cum, U):
    c = np.ascontiguousarray(cum, dtype=np.uint64)
    return int(lib().orc_fix_choose(_p(c), c.size, int(U)))


def fair_draws(prob, theta, lnw, n_draws, seed):
    """Fair draws from the weighted samples (theta [n][6], lnw [n]): sample indices,
    their theta, and each draw's time bin and time from the sample's per-bin ln L
    (evaluated here in float64).  Returns (idx, theta, j, t)."""
    P = _as_problem(prob)
    w = np.ascontiguousarray(lnw, dtype=np.float64)
    idx = np.empty(int(n_draws), np.int64)
    Ut = np.empty(int(n_draws), np.uint64)
    if lib().orc_fair_draws(_p(w), w.size, int(seed), int(n_draws), _p(idx), _p(Ut)) != 0:
        raise ValueError("no finite log-weight")
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(-1, 6)[idx])
    _, bins, _ = lnL(P, th, want_bins=True)
    j = np.empty(int(n_draws), np.int64)
    for d in range(int(n_draws)):
        row = np.ascontiguousarray(bins[d])
        j[d] = lib().orc_fair_time_bin(_p(row), row.size, int(Ut[d]))
    t_lo, t_hi = P.s.t_lo, P.s.t_hi
    step = (t_hi - t_lo) / (P.n_t - 1) if P.n_t > 1 else 0.0
    t = t_lo + j * step
    return idx, th, j, t


def ln_dist_marg(a, b, d_ref, d_min, d_max):
    """ln of the distance-marginal likelihood of one bin with data term a and template
    term b at D = D_ref (prior D^2 on [d_min, d_max])."""
    return lib().orc_ln_dist_marg(float(d_ref), float(d_min), float(d_max), float(a), float(b))


def num_threads() -> int:
    return lib().orc_num_threads()
