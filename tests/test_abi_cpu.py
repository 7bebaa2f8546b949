"""The C-ABI library builds, loads and exports every declared entry point; the
host-side validation rejects bad configurations before any device work.
CPU only: no call here launches a kernel."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import ile_synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import paper_2505_11655_gb300 as G
    G.load(build_if_missing=True)
    return G


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "rift_ile.h")).read()
    return sorted(set(re.findall(r"\b(rift_(?:ile|srv|batch)_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 19
    L = C.CDLL(lib._LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(lib.EXPORTED)


def test_strerror_names_every_code(lib):
    for code in range(0, -8, -1):
        assert lib.strerror(code) not in ("", "unknown status")
    assert lib.strerror(-99) == "unknown status"


def _cfg(lib, prob, **over):
    keep = dict(t=np.ascontiguousarray(prob.det_tensor), p=np.ascontiguousarray(prob.det_pos),
                lm=np.ascontiguousarray(prob.lm, np.int32), t0=np.ascontiguousarray(prob.q_t0))
    vals = dict(n_det=prob.n_det, det_tensor=keep["t"].ctypes.data, det_pos_m=keep["p"].ctypes.data, gmst_rad=prob.gmst,
                n_modes=prob.n_modes, lm=keep["lm"].ctypes.data, fs_hz=prob.fs, n_q=prob.n_q,
                q_t0_s=keep["t0"].ctypes.data, t_lo_s=prob.t_lo, t_hi_s=prob.t_hi, n_t=prob.n_t,
                d_ref_mpc=prob.d_ref, d_min_mpc=prob.d_min, d_max_mpc=prob.d_max, quad_norm=0, precision=1,
                n_bins=64, adapt_floor=0.1, adapt_temper=1.0, seed=1, max_samples=1000)
    vals.update(over)
    cfg = lib.rift_ile_config(**vals)
    return cfg, keep


def _create_rc(lib, cfg):
    h = C.c_void_p()
    return lib.load().rift_ile_create(C.byref(cfg), None, C.byref(h))


@pytest.mark.parametrize("field,value", [
    ("n_det", 0), ("n_det", 5), ("n_modes", 0), ("n_modes", 33), ("fs_hz", 0.0), ("n_q", 1), ("n_t", 0),
    ("d_ref_mpc", 0.0), ("d_min_mpc", 2000.0), ("quad_norm", 2), ("precision", 7), ("n_bins", 1), ("distance_marg", 2),
    ("n_bins", 4096), ("adapt_floor", 1.0), ("adapt_temper", 0.0), ("max_samples", 0),
])
def test_invalid_config_rejected(lib, field, value):
    prob = S.plain_fp64_problem()
    cfg, keep = _cfg(lib, prob, **{field: value})
    assert _create_rc(lib, cfg) == lib.RIFT_EINVAL


def test_bad_modes_rejected(lib):
    prob = S.plain_fp64_problem()
    for lm in ([[2, 2], [2, 2]], [[1, 0], [2, 2]], [[2, 3], [2, 2]], [[7, 0], [2, 2]]):
        arr = np.array(lm, np.int32)
        cfg, keep = _cfg(lib, prob, lm=arr.ctypes.data)
        assert _create_rc(lib, cfg) == lib.RIFT_EINVAL


def test_window_violation_is_erange(lib):
    """The grid plus the largest light-travel delay must map inside the Q window."""
    prob = S.plain_fp64_problem()
    t0 = np.array([-0.06, -0.1])
    cfg, keep = _cfg(lib, prob, q_t0_s=t0.ctypes.data)
    assert _create_rc(lib, cfg) == lib.RIFT_ERANGE
    cfg, keep = _cfg(lib, prob, t_hi_s=0.08)
    assert _create_rc(lib, cfg) == lib.RIFT_ERANGE


def test_footprint_is_host_only_and_grows_with_samples(lib):
    """rift_ile_footprint validates and sizes a configuration without any CUDA call."""
    prob = S.single_large_problem()
    cfg, keep = _cfg(lib, prob, max_samples=1000)
    small = lib.rift_ile_footprint(cfg)
    cfg2, keep2 = _cfg(lib, prob, max_samples=1_000_000)
    big = lib.rift_ile_footprint(cfg2)
    assert 0 < small < big
    assert big - small >= 88 * (1_000_000 - 1000)   # per-sample buffers
    bad, keep3 = _cfg(lib, prob, n_det=0)
    assert lib.rift_ile_footprint(bad) == -1


def test_server_rejects_bad_config(lib):
    L = lib.load()
    h = C.c_void_p()
    for budget, slots in ((0, 4), (1 << 30, 0), (1 << 30, 65)):
        cfg = lib.rift_srv_config(budget, slots)
        assert L.rift_srv_create(C.byref(cfg), C.byref(h)) == lib.RIFT_EINVAL


def test_valid_config_without_gpu_is_ecuda(lib):
    """A valid configuration gets past validation; with no GPU the create call
    reports a CUDA failure instead of falling back to anything."""
    pytest.importorskip("torch")
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    prob = S.plain_fp64_problem()
    cfg, keep = _cfg(lib, prob)
    assert _create_rc(lib, cfg) == lib.RIFT_ECUDA


def test_binding_refuses_missing_library(tmp_path, monkeypatch):
    import paper_2505_11655_gb300 as G
    monkeypatch.setattr(G, "_lib", None)
    monkeypatch.setattr(G, "_LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        G.load()


def test_batch_rejects_bad_arguments(lib):
    """rift_batch_create validates its arguments before any CUDA call."""
    L = lib.load()
    b = C.c_void_p()
    it = (C.c_int32 * 2)(1, 1)
    ns = (C.c_int64 * 2)(100, 100)
    hs = (C.c_void_p * 2)(None, None)
    assert L.rift_batch_create(hs, 2, it, ns, None, C.byref(b)) == lib.RIFT_EINVAL
    assert L.rift_batch_create(hs, 0, it, ns, None, C.byref(b)) == lib.RIFT_EINVAL
    assert L.rift_batch_create(None, 2, it, ns, None, C.byref(b)) == lib.RIFT_EINVAL
    assert L.rift_batch_run(None, None) == lib.RIFT_EINVAL
    assert L.rift_batch_kernel_launches(None) == -1
    assert L.rift_ile_get_plan(None, None, None) == lib.RIFT_EINVAL
