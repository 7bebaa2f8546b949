"""Python binding of the GB300 ILE library (arXiv:2505.11655 hot path).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``librift_ile.so`` behind the C ABI declared in
``include/rift_ile.h``.  The functions here carry the same names as the C
entry points.  Host arrays are numpy arrays; device arrays are torch CUDA
tensors (their ``data_ptr()`` is passed through), torch being used for device
memory and streams only.

There is no CPU fallback: importing the binding without the built library
raises, and so does any call that the library rejects.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB as _LIB_PATH
from .build import build as _build

RIFT_OK, RIFT_EINVAL, RIFT_ENOMEM, RIFT_ECUDA = 0, -1, -2, -3
RIFT_ERANGE, RIFT_ENONFINITE, RIFT_ETIMEOUT, RIFT_ESTATE = -4, -5, -6, -7
RIFT_MEM_HOST, RIFT_MEM_DEVICE = 0, 1
RIFT_QUAD_QUARTER, RIFT_QUAD_HALF = 0, 1
RIFT_FP64, RIFT_FP32, RIFT_MIXED = 0, 1, 2
RIFT_MAX_ITER = 64
RIFT_KERNEL_FP64, RIFT_KERNEL_CUDA_CORE, RIFT_KERNEL_TENSOR = 0, 1, 2

EXPORTED = ["rift_ile_create", "rift_ile_set_overlaps", "rift_ile_set_waveforms", "rift_ile_get_overlaps", "rift_ile_eval", "rift_ile_coeffs", "rift_ile_marginalize",
            "rift_ile_adapt", "rift_ile_last_batch", "rift_ile_get_state", "rift_ile_set_state",
            "rift_ile_get_sampler", "rift_ile_kernel_launches", "rift_ile_reduce_noalloc", "rift_ile_footprint",
            "rift_ile_get_plan", "rift_ile_peak_rate", "rift_ile_wait_selftest", "rift_ile_fair_draws", "rift_ile_av", "rift_ile_av_info", "rift_ile_portfolio", "rift_ile_portfolio_info", "rift_ile_portfolio_gmm", "rift_ile_destroy", "rift_ile_strerror", "rift_batch_create", "rift_batch_run",
            "rift_batch_kernel_launches", "rift_batch_destroy", "rift_srv_create", "rift_srv_submit", "rift_srv_poll",
            "rift_srv_pending", "rift_srv_destroy"]


class RiftError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


class rift_ile_config(C.Structure):
    _fields_ = [
        ("n_det", C.c_int32), ("det_tensor", C.c_void_p), ("det_pos_m", C.c_void_p), ("gmst_rad", C.c_double),
        ("n_modes", C.c_int32), ("lm", C.c_void_p), ("fs_hz", C.c_double), ("n_q", C.c_int32),
        ("q_t0_s", C.c_void_p), ("t_lo_s", C.c_double), ("t_hi_s", C.c_double), ("n_t", C.c_int32),
        ("d_ref_mpc", C.c_double), ("d_min_mpc", C.c_double), ("d_max_mpc", C.c_double),
        ("quad_norm", C.c_int32), ("precision", C.c_int32), ("n_bins", C.c_int32), ("adapt_floor", C.c_double),
        ("adapt_temper", C.c_double), ("seed", C.c_uint64), ("max_samples", C.c_int64),
        ("distance_marg", C.c_int32),
    ]


RIFT_MEMBER_HIST = 1
RIFT_MEMBER_AV = 2
RIFT_MEMBER_GMM = 4
RIFT_GMM_MAX_COMPONENTS = 16


class rift_portfolio_config(C.Structure):
    _fields_ = [("members", C.c_int32), ("av_start", C.c_int32), ("gmm_start", C.c_int32),
                ("gmm_components", C.c_int32), ("adapt_weights", C.c_int32), ("reserved", C.c_int32),
                ("w_init", C.c_double * 3), ("p_thr", C.c_double), ("n_min_star", C.c_int64),
                ("capacity", C.c_int64)]


class rift_portfolio_info(C.Structure):
    _fields_ = [("iteration", C.c_int32), ("active", C.c_int32 * 3), ("frozen", C.c_int32 * 3),
                ("reserved", C.c_int32), ("W_last", C.c_double * 3), ("W_next", C.c_double * 3),
                ("n_ess", C.c_double * 3), ("n_drawn", C.c_int64 * 3)]

    def as_dict(self):
        return dict(iteration=self.iteration, active=list(self.active), frozen=list(self.frozen),
                    W_last=list(self.W_last), W_next=list(self.W_next), n_ess=list(self.n_ess),
                    n_drawn=list(self.n_drawn))


class rift_ile_result(C.Structure):
    _fields_ = [
        ("lnZ", C.c_double), ("sigma_lnZ", C.c_double), ("n_eff", C.c_double), ("n_ess", C.c_double),
        ("lnL_max", C.c_double), ("n_total", C.c_int64), ("n_iter", C.c_int32), ("status", C.c_int32),
        ("lnZ_iter", C.c_double * RIFT_MAX_ITER), ("sigma_iter", C.c_double * RIFT_MAX_ITER),
        ("n_eff_iter", C.c_double * RIFT_MAX_ITER), ("n_ess_iter", C.c_double * RIFT_MAX_ITER),
        ("time_ms", C.c_double * 4),
    ]

    def as_dict(self):
        n = self.n_iter
        return dict(lnZ=self.lnZ, sigma_lnZ=self.sigma_lnZ, n_eff=self.n_eff, n_ess=self.n_ess,
                    lnL_max=self.lnL_max, n_total=self.n_total, n_iter=n, status=self.status,
                    lnZ_iter=list(self.lnZ_iter[:n]), sigma_iter=list(self.sigma_iter[:n]),
                    n_eff_iter=list(self.n_eff_iter[:n]), n_ess_iter=list(self.n_ess_iter[:n]),
                    time_ms=list(self.time_ms))


class rift_srv_config(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("max_slots", C.c_int32)]


class rift_srv_request(C.Structure):
    _fields_ = [("cfg", C.POINTER(rift_ile_config)), ("Q", C.c_void_p), ("U", C.c_void_p), ("V", C.c_void_p),
                ("n_iter", C.c_int32), ("n_per_iter", C.c_int64), ("tag", C.c_uint64)]


class rift_srv_completion(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("status", C.c_int32), ("result", rift_ile_result),
                ("t_submit_ms", C.c_double), ("t_admit_ms", C.c_double), ("t_done_ms", C.c_double)]


_lib = None


def load(build_if_missing: bool = False):
    """Load librift_ile.so (optionally building it first).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build()
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"CUDA library not built: {_LIB_PATH} (run paper_2505_11655_gb300/build.py)")
    L = C.CDLL(_LIB_PATH)
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    L.rift_ile_create.argtypes = [C.POINTER(rift_ile_config), vp, C.POINTER(vp)]
    L.rift_ile_set_overlaps.argtypes = [vp, vp, vp, vp, C.c_int]
    L.rift_ile_eval.argtypes = [vp, vp, i64, C.c_int, vp, vp]
    L.rift_ile_coeffs.argtypes = [vp, vp, i64, C.c_int, vp, vp, vp]
    L.rift_ile_marginalize.argtypes = [vp, i64, C.POINTER(rift_ile_result)]
    L.rift_ile_adapt.argtypes = [vp, i32, i64, C.POINTER(rift_ile_result)]
    L.rift_ile_last_batch.argtypes = [vp, C.c_int, vp, vp, vp, vp, C.POINTER(i64)]
    L.rift_ile_get_state.argtypes = [vp, vp, C.POINTER(C.c_size_t)]
    L.rift_ile_set_state.argtypes = [vp, vp, C.c_size_t]
    L.rift_ile_get_sampler.argtypes = [vp, vp]
    L.rift_ile_reduce_noalloc.argtypes = [vp, vp, i64, vp, vp]
    L.rift_ile_footprint.argtypes = [C.POINTER(rift_ile_config)]
    L.rift_ile_footprint.restype = C.c_int64
    L.rift_srv_create.argtypes = [C.POINTER(rift_srv_config), C.POINTER(vp)]
    L.rift_srv_submit.argtypes = [vp, C.POINTER(rift_srv_request)]
    L.rift_srv_poll.argtypes = [vp, C.POINTER(rift_srv_completion), C.c_int32, C.c_int32, C.POINTER(C.c_int32)]
    L.rift_srv_pending.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    L.rift_srv_destroy.argtypes = [vp]
    L.rift_srv_destroy.restype = None
    L.rift_ile_get_plan.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
    L.rift_ile_wait_selftest.argtypes = [vp, i64]
    L.rift_ile_peak_rate.argtypes = [i32, C.POINTER(C.c_double)]
    L.rift_ile_fair_draws.argtypes = [vp, i64, C.c_uint64, C.c_int, vp, vp, vp]
    L.rift_ile_set_waveforms.argtypes = [vp, i32, vp, vp, vp, vp, C.c_int]
    L.rift_ile_get_overlaps.argtypes = [vp, vp, vp, vp, C.c_int]
    L.rift_ile_av.argtypes = [vp, i32, i64, C.c_double, i64, i64, i32, C.POINTER(rift_ile_result)]
    L.rift_ile_av_info.argtypes = [vp, C.POINTER(i32), C.POINTER(i64), C.POINTER(i64), C.POINTER(C.c_double)]
    L.rift_ile_portfolio.argtypes = [vp, i32, i64, C.POINTER(rift_portfolio_config), i32, C.POINTER(rift_ile_result)]
    L.rift_ile_portfolio_info.argtypes = [vp, C.POINTER(rift_portfolio_info)]
    L.rift_ile_portfolio_gmm.argtypes = [vp, i32, C.POINTER(i32), vp, vp, vp]
    L.rift_batch_create.argtypes = [C.POINTER(vp), i32, C.POINTER(i32), C.POINTER(i64), vp, C.POINTER(vp)]
    L.rift_batch_run.argtypes = [vp, C.POINTER(rift_ile_result)]
    L.rift_batch_kernel_launches.argtypes = [vp]
    L.rift_batch_kernel_launches.restype = C.c_int64
    L.rift_batch_destroy.argtypes = [vp]
    L.rift_batch_destroy.restype = None
    L.rift_ile_kernel_launches.argtypes = [vp]
    L.rift_ile_kernel_launches.restype = C.c_int64
    L.rift_ile_destroy.argtypes = [vp]
    L.rift_ile_destroy.restype = None
    L.rift_ile_strerror.argtypes = [C.c_int]
    L.rift_ile_strerror.restype = C.c_char_p
    for name in EXPORTED:
        if name not in ("rift_ile_destroy", "rift_ile_strerror", "rift_ile_kernel_launches", "rift_ile_footprint",
                        "rift_srv_destroy"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def strerror(code: int) -> str:
    return load().rift_ile_strerror(int(code)).decode()


def _check(rc, what):
    if rc != RIFT_OK:
        raise RiftError(rc, what)


def _ptr(a):
    """Address of a numpy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported buffer type {type(a)}")


def _mem(a):
    if isinstance(a, np.ndarray):
        return RIFT_MEM_HOST
    if hasattr(a, "is_cuda"):
        if not a.is_cuda:
            raise ValueError("torch tensors must be on the GPU; pass numpy arrays for host memory")
        return RIFT_MEM_DEVICE
    raise TypeError(f"unsupported buffer type {type(a)}")


# ---------------------------------------------------------------------------------- C-named calls

def rift_ile_create(cfg: rift_ile_config, stream=None):
    h = C.c_void_p()
    st = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    _check(load().rift_ile_create(C.byref(cfg), st, C.byref(h)), "rift_ile_create")
    return h


def rift_ile_set_overlaps(h, Q, U, V):
    mem = _mem(Q)
    if _mem(U) != mem or _mem(V) != mem:
        raise ValueError("Q, U, V must live in the same memory")
    _check(load().rift_ile_set_overlaps(h, _ptr(Q), _ptr(U), _ptr(V), mem), "rift_ile_set_overlaps")


def rift_ile_eval(h, theta, n, lnL_tmarg, lnL_t=None):
    _check(load().rift_ile_eval(h, _ptr(theta), int(n), _mem(theta), _ptr(lnL_tmarg), _ptr(lnL_t)), "rift_ile_eval")


def rift_ile_coeffs(h, theta, n, c=None, dt=None, quad=None):
    _check(load().rift_ile_coeffs(h, _ptr(theta), int(n), _mem(theta), _ptr(c), _ptr(dt), _ptr(quad)),
           "rift_ile_coeffs")


def rift_ile_marginalize(h, n_samples):
    r = rift_ile_result()
    _check(load().rift_ile_marginalize(h, int(n_samples), C.byref(r)), "rift_ile_marginalize")
    return r


def rift_ile_adapt(h, n_iter, n_per_iter):
    r = rift_ile_result()
    _check(load().rift_ile_adapt(h, int(n_iter), int(n_per_iter), C.byref(r)), "rift_ile_adapt")
    return r


def rift_ile_last_batch(h, theta=None, lnp_minus_lnps=None, lnL_tmarg=None, lnw=None, mem=RIFT_MEM_HOST):
    n = C.c_int64()
    _check(load().rift_ile_last_batch(h, mem, _ptr(theta), _ptr(lnp_minus_lnps), _ptr(lnL_tmarg), _ptr(lnw),
                                      C.byref(n)), "rift_ile_last_batch")
    return n.value


def rift_ile_get_state(h) -> bytes:
    n = C.c_size_t()
    _check(load().rift_ile_get_state(h, None, C.byref(n)), "rift_ile_get_state")
    buf = C.create_string_buffer(n.value)
    _check(load().rift_ile_get_state(h, buf, C.byref(n)), "rift_ile_get_state")
    return buf.raw[: n.value]


def rift_ile_set_state(h, blob: bytes):
    _check(load().rift_ile_set_state(h, blob, len(blob)), "rift_ile_set_state")


def rift_ile_get_sampler(h, n_bins):
    P = np.empty((6, n_bins))
    _check(load().rift_ile_get_sampler(h, _ptr(P)), "rift_ile_get_sampler")
    return P


def rift_ile_reduce_noalloc(lnw, n, out, lnL=None, stream=None):
    """Reduction of device log-weights into device out[8] without allocating."""
    st = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    _check(load().rift_ile_reduce_noalloc(_ptr(lnw), _ptr(lnL), int(n), _ptr(out), st), "rift_ile_reduce_noalloc")


def rift_ile_footprint(cfg):
    return int(load().rift_ile_footprint(C.byref(cfg)))


def rift_srv_create(hbm_budget_bytes, max_slots):
    h = C.c_void_p()
    cfg = rift_srv_config(int(hbm_budget_bytes), int(max_slots))
    _check(load().rift_srv_create(C.byref(cfg), C.byref(h)), "rift_srv_create")
    return h


def rift_srv_submit(srv, cfg, Q, U, V, n_iter, n_per_iter, tag):
    req = rift_srv_request(C.pointer(cfg), _ptr(Q), _ptr(U), _ptr(V), int(n_iter), int(n_per_iter), int(tag))
    _check(load().rift_srv_submit(srv, C.byref(req)), "rift_srv_submit")


def rift_srv_poll(srv, max_n=256, timeout_ms=0):
    buf = (rift_srv_completion * max_n)()
    n = C.c_int32()
    _check(load().rift_srv_poll(srv, buf, max_n, int(timeout_ms), C.byref(n)), "rift_srv_poll")
    return [buf[i] for i in range(n.value)]


def rift_srv_pending(srv):
    q, a = C.c_int32(), C.c_int32()
    _check(load().rift_srv_pending(srv, C.byref(q), C.byref(a)), "rift_srv_pending")
    return q.value, a.value


def rift_srv_destroy(srv):
    if srv:
        load().rift_srv_destroy(srv)


def rift_ile_kernel_launches(h):
    return int(load().rift_ile_kernel_launches(h))


def rift_ile_wait_selftest(h, limit_ns):
    """Status of one bounded wait that runs out (RIFT_ETIMEOUT when the failure path works)."""
    return int(load().rift_ile_wait_selftest(h, int(limit_ns)))


RIFT_PEAK_FP32_FMA, RIFT_PEAK_TC_F16_N128, RIFT_PEAK_TC_F16_N256, RIFT_PEAK_EX2, RIFT_PEAK_FP64_FMA = 0, 1, 2, 3, 4


def rift_ile_peak_rate(what):
    """Measured peak rate (tera-operations/s) of a unit: RIFT_PEAK_FP32_FMA, _TC_F16_N128,
    _TC_F16_N256, _EX2 (exponentials/s) or _FP64_FMA."""
    v = C.c_double()
    _check(load().rift_ile_peak_rate(int(what), C.byref(v)), "rift_ile_peak_rate")
    return v.value


def rift_ile_get_plan(h):
    k, c = C.c_int32(), C.c_int32()
    _check(load().rift_ile_get_plan(h, C.byref(k), C.byref(c)), "rift_ile_get_plan")
    return k.value, c.value


def rift_ile_set_waveforms(h, freqs, hlm, data, weights):
    _check(load().rift_ile_set_waveforms(h, int(freqs.shape[0]), _ptr(freqs), _ptr(hlm), _ptr(data), _ptr(weights),
                                         _mem(freqs)), "rift_ile_set_waveforms")


def rift_ile_get_overlaps(h, Q=None, U=None, V=None):
    bufs = [b for b in (Q, U, V) if b is not None]
    mem = _mem(bufs[0]) if bufs else RIFT_MEM_HOST
    _check(load().rift_ile_get_overlaps(h, _ptr(Q), _ptr(U), _ptr(V), mem), "rift_ile_get_overlaps")


def rift_ile_fair_draws(h, n_draws, seed, theta=None, t=None, index=None):
    bufs = [b for b in (theta, t, index) if b is not None]
    mem = _mem(bufs[0]) if bufs else RIFT_MEM_HOST
    _check(load().rift_ile_fair_draws(h, int(n_draws), int(seed), mem, _ptr(theta), _ptr(t), _ptr(index)),
           "rift_ile_fair_draws")


def rift_ile_av(h, n_iter, n_per_iter, p_thr, n_min_star, capacity, restart):
    r = rift_ile_result()
    _check(load().rift_ile_av(h, int(n_iter), int(n_per_iter), float(p_thr), int(n_min_star), int(capacity),
                              int(restart), C.byref(r)), "rift_ile_av")
    return r


def rift_ile_portfolio(h, n_iter, n_per_iter, cfg, restart):
    r = rift_ile_result()
    _check(load().rift_ile_portfolio(h, int(n_iter), int(n_per_iter), C.byref(cfg), int(restart), C.byref(r)),
           "rift_ile_portfolio")
    return r


def rift_ile_portfolio_info(h):
    info = rift_portfolio_info()
    _check(load().rift_ile_portfolio_info(h, C.byref(info)), "rift_ile_portfolio_info")
    return info.as_dict()


def rift_ile_portfolio_gmm(h):
    """The GMM member's (pi [C], mu [C][6], sig [C][6])."""
    k = RIFT_GMM_MAX_COMPONENTS
    pi, mu, sig = np.zeros(k), np.zeros((k, 6)), np.zeros((k, 6))
    nc = C.c_int32(0)
    _check(load().rift_ile_portfolio_gmm(h, k, C.byref(nc), pi.ctypes.data, mu.ctypes.data, sig.ctypes.data),
           "rift_ile_portfolio_gmm")
    c = nc.value
    return pi[:c].copy(), mu[:c].copy(), sig[:c].copy()


def rift_ile_av_info(h):
    lv, nc, nl, V = C.c_int32(), C.c_int64(), C.c_int64(), C.c_double()
    _check(load().rift_ile_av_info(h, C.byref(lv), C.byref(nc), C.byref(nl), C.byref(V)), "rift_ile_av_info")
    return dict(level=lv.value, n_cells=nc.value, n_live=nl.value, V=V.value)


def rift_batch_create(handles, n_iter, n_per_iter, stream=None):
    n = len(handles)
    hs = (C.c_void_p * n)(*handles)
    it = (C.c_int32 * n)(*[int(x) for x in n_iter])
    ns = (C.c_int64 * n)(*[int(x) for x in n_per_iter])
    b = C.c_void_p()
    st = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    _check(load().rift_batch_create(hs, n, it, ns, st, C.byref(b)), "rift_batch_create")
    return b


def rift_batch_run(b, n):
    out = (rift_ile_result * n)()
    rc = load().rift_batch_run(b, out)
    if rc not in (RIFT_OK, RIFT_ERANGE, RIFT_ENONFINITE, RIFT_ETIMEOUT):
        raise RiftError(rc, "rift_batch_run")
    return list(out), rc


def rift_batch_kernel_launches(b):
    return int(load().rift_batch_kernel_launches(b))


def rift_batch_destroy(b):
    if b:
        load().rift_batch_destroy(b)


def rift_ile_destroy(h):
    if h:
        load().rift_ile_destroy(h)


def rift_ile_strerror(code):
    return strerror(code)


# ---------------------------------------------------------------------------------- convenience

def make_config(prob, precision=RIFT_FP32, max_samples=1 << 20, n_bins=64, adapt_floor=0.1, adapt_temper=1.0,
                seed=1, distance_marg=False):
    """rift_ile_config for a problem (attributes of ile_synth.Problem) and the host
    arrays it points at (keep the returned dict alive as long as the config)."""
    keep = dict(
        det_tensor=np.ascontiguousarray(prob.det_tensor, np.float64),
        det_pos=np.ascontiguousarray(prob.det_pos, np.float64),
        lm=np.ascontiguousarray(prob.lm, np.int32),
        q_t0=np.ascontiguousarray(prob.q_t0, np.float64),
    )
    cfg = rift_ile_config(
        keep["det_tensor"].shape[0], _ptr(keep["det_tensor"]), _ptr(keep["det_pos"]), float(prob.gmst),
        keep["lm"].shape[0], _ptr(keep["lm"]), float(prob.fs), int(prob.n_q), _ptr(keep["q_t0"]), float(prob.t_lo),
        float(prob.t_hi), int(prob.n_t), float(prob.d_ref), float(prob.d_min), float(prob.d_max),
        int(prob.quad_norm), int(precision), int(n_bins), float(adapt_floor), float(adapt_temper), int(seed),
        int(max_samples), int(bool(distance_marg)))
    return cfg, keep


class Server:
    """Request loop for many solves (rift_srv_*): submit problems as they arrive,
    poll completions with their submit/admit/done times."""

    def __init__(self, hbm_budget_bytes=32 << 30, max_slots=8):
        self.h = rift_srv_create(hbm_budget_bytes, max_slots)
        self._keep = []

    def submit(self, prob, n_iter, n_per_iter, tag, precision=RIFT_FP32, n_bins=64, seed=1, distance_marg=False):
        cfg, keep = make_config(prob, precision, max_samples=n_per_iter, n_bins=n_bins, seed=seed,
                                distance_marg=distance_marg)
        arrs = [np.ascontiguousarray(x, np.complex128) for x in (prob.Q, prob.U, prob.V)]
        rift_srv_submit(self.h, cfg, arrs[0], arrs[1], arrs[2], n_iter, n_per_iter, tag)

    def poll(self, max_n=256, timeout_ms=0):
        out = []
        for c in rift_srv_poll(self.h, max_n, timeout_ms):
            d = c.result.as_dict()
            d.update(tag=c.tag, status=c.status, t_submit_ms=c.t_submit_ms, t_admit_ms=c.t_admit_ms,
                     t_done_ms=c.t_done_ms)
            out.append(d)
        return out

    def pending(self):
        return rift_srv_pending(self.h)

    def drain(self, n_expected, timeout_s=600.0):
        """Poll until n_expected completions arrived (or the timeout)."""
        import time
        got, t0 = [], time.time()
        while len(got) < n_expected and time.time() - t0 < timeout_s:
            got += self.poll(256, 100)
        return got

    def close(self):
        if getattr(self, "h", None):
            rift_srv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Many solves as one CUDA graph (rift_batch_*): ``solves`` are ILE objects with
    their overlaps set, each run continues every solve's adaptive sequence."""

    def __init__(self, solves, n_iter, n_per_iter, stream=None):
        self.solves = list(solves)   # keep the handles alive
        self.h = rift_batch_create([s.h for s in self.solves], n_iter, n_per_iter, stream)

    def run(self):
        """Results (dicts, one per solve, each with its own status) and the first
        failing status (0 if none)."""
        res, rc = rift_batch_run(self.h, len(self.solves))
        return [r.as_dict() for r in res], rc

    def kernel_launches(self):
        return rift_batch_kernel_launches(self.h)

    def close(self):
        if getattr(self, "h", None):
            rift_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class ILE:
    """One handle for one intrinsic point.  ``prob`` carries the problem's host
    arrays (the attributes of ``ile_synth.Problem``)."""

    def __init__(self, prob, precision=RIFT_FP32, max_samples=1 << 20, n_bins=64, adapt_floor=0.1,
                 adapt_temper=1.0, seed=1, stream=None, set_overlaps=True, distance_marg=False):
        self._keep = dict(
            det_tensor=np.ascontiguousarray(prob.det_tensor, np.float64),
            det_pos=np.ascontiguousarray(prob.det_pos, np.float64),
            lm=np.ascontiguousarray(prob.lm, np.int32),
            q_t0=np.ascontiguousarray(prob.q_t0, np.float64),
        )
        k = self._keep
        self.n_det, self.n_modes, self.n_t, self.n_bins = k["det_tensor"].shape[0], k["lm"].shape[0], prob.n_t, n_bins
        self.cfg = rift_ile_config(
            self.n_det, _ptr(k["det_tensor"]), _ptr(k["det_pos"]), float(prob.gmst), self.n_modes, _ptr(k["lm"]),
            float(prob.fs), int(prob.n_q), _ptr(k["q_t0"]), float(prob.t_lo), float(prob.t_hi), int(prob.n_t),
            float(prob.d_ref), float(prob.d_min), float(prob.d_max), int(prob.quad_norm), int(precision),
            int(n_bins), float(adapt_floor), float(adapt_temper), int(seed), int(max_samples),
            int(bool(distance_marg)))
        self.h = rift_ile_create(self.cfg, stream)
        if set_overlaps:
            self.set_overlaps(prob.Q, prob.U, prob.V)

    def set_overlaps(self, Q, U, V):
        if isinstance(Q, np.ndarray):
            Q, U, V = (np.ascontiguousarray(x, np.complex128) for x in (Q, U, V))
        rift_ile_set_overlaps(self.h, Q, U, V)

    def set_waveforms(self, freqs, hlm, data, weights):
        """Q, U, V computed on the device from frequency-domain inputs (numpy or torch)."""
        if isinstance(freqs, np.ndarray):
            freqs = np.ascontiguousarray(freqs, np.float64)
            hlm, data = (np.ascontiguousarray(x, np.complex128) for x in (hlm, data))
            weights = np.ascontiguousarray(weights, np.float64)
        rift_ile_set_waveforms(self.h, freqs, hlm, data, weights)

    def get_overlaps(self, n_q):
        Q = np.empty((self.n_det, self.n_modes, n_q), np.complex128)
        U = np.empty((self.n_det, self.n_modes, self.n_modes), np.complex128)
        V = np.empty_like(U)
        rift_ile_get_overlaps(self.h, Q, U, V)
        return Q, U, V

    def eval(self, theta, want_bins=False):
        if isinstance(theta, np.ndarray):
            th = np.ascontiguousarray(theta, np.float64).reshape(-1, 6)
            out = np.empty(th.shape[0])
            bins = np.empty((th.shape[0], self.n_t)) if want_bins else None
        else:
            import torch
            th = theta.reshape(-1, 6).contiguous()
            out = torch.empty(th.shape[0], dtype=torch.float64, device=th.device)
            bins = torch.empty((th.shape[0], self.n_t), dtype=torch.float64, device=th.device) if want_bins else None
        rift_ile_eval(self.h, th, th.shape[0], out, bins)
        return (out, bins) if want_bins else out

    def coeffs(self, theta):
        th = np.ascontiguousarray(theta, np.float64).reshape(-1, 6)
        n = th.shape[0]
        c = np.empty((n, self.n_det, self.n_modes), np.complex128)
        dt = np.empty((n, self.n_det))
        quad = np.empty(n)
        rift_ile_coeffs(self.h, th, n, c, dt, quad)
        return c, dt, quad

    def marginalize(self, n):
        return rift_ile_marginalize(self.h, n).as_dict()

    def adapt(self, n_iter, n_per_iter):
        return rift_ile_adapt(self.h, n_iter, n_per_iter).as_dict()

    def last_batch(self, n):
        th, lr, ll, lw = np.empty((n, 6)), np.empty(n), np.empty(n), np.empty(n)
        m = rift_ile_last_batch(self.h, th, lr, ll, lw)
        return th[:m], lr[:m], ll[:m], lw[:m]

    def kernel_launches(self):
        return rift_ile_kernel_launches(self.h)

    def av(self, n_iter, n_per_iter, p_thr=0.9999, n_min_star=1000, capacity=None, restart=False):
        """Adaptive-volume iterations (rift_ile_av); capacity defaults to 4 n_per_iter."""
        cap = 4 * n_per_iter if capacity is None else capacity
        return rift_ile_av(self.h, n_iter, n_per_iter, p_thr, n_min_star, cap, 1 if restart else 0).as_dict()

    def av_info(self):
        return rift_ile_av_info(self.h)

    def portfolio(self, n_iter, n_per_iter, members=RIFT_MEMBER_HIST | RIFT_MEMBER_AV, av_start=0, gmm_start=0,
                  gmm_components=4, adapt_weights=True, w_init=None, p_thr=0.9999, n_min_star=1000, capacity=None,
                  restart=False):
        """Portfolio iterations over {histogram, AV, GMM} (rift_ile_portfolio); capacity
        defaults to 4 n_per_iter, w_init to equal weights over the members."""
        if w_init is None:
            w_init = [1.0 if (members >> m) & 1 else 0.0 for m in range(3)]
        w = [float(x) for x in w_init] + [0.0] * (3 - len(w_init))
        cfg = rift_portfolio_config(int(members), int(av_start), int(gmm_start), int(gmm_components),
                                    1 if adapt_weights else 0, 0, (C.c_double * 3)(*w), float(p_thr), int(n_min_star),
                                    int(capacity if capacity is not None else 4 * n_per_iter))
        return rift_ile_portfolio(self.h, n_iter, n_per_iter, cfg, 1 if restart else 0).as_dict()

    def portfolio_info(self):
        return rift_ile_portfolio_info(self.h)

    def portfolio_gmm(self):
        return rift_ile_portfolio_gmm(self.h)

    def fair_draws(self, n_draws, seed=1):
        """Fair draws from the most recent batch: (theta [n][6], t [n], index [n])."""
        th, t, idx = np.empty((n_draws, 6)), np.empty(n_draws), np.empty(n_draws, np.int64)
        rift_ile_fair_draws(self.h, n_draws, seed, th, t, idx)
        return th, t, idx

    def plan(self):
        """(likelihood kernel: RIFT_KERNEL_*, samples per sky cell) of the last batch."""
        return rift_ile_get_plan(self.h)

    def sampler(self):
        return rift_ile_get_sampler(self.h, self.n_bins)

    def get_state(self):
        return rift_ile_get_state(self.h)

    def set_state(self, blob):
        rift_ile_set_state(self.h, blob)

    def close(self):
        if getattr(self, "h", None):
            rift_ile_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
