"""GPU parity of the tensor-core likelihood kernel across problem shapes: the
tensor-memory layout (accumulators, coefficient operand at 256 + (2k + part) kp/2,
template products at 64 k), the shared-memory layout and the step schedule all
depend on the detector count K, the padded mode width kp and the time grid, so the
kernel is compared with the float64 oracle (and with the CUDA-core kernel) on
K = 1, 2, 4 and kp = 16, 32, 48, 64, at batch sizes spanning several 128-sample tiles
and a ragged tail."""
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


FP32_TOL = 1e-3   # |d ln L| on every sample for the float32 path


def clustered(n, seed, center=(1.0, 0.3), width=0.06):
    th = S.prior_samples(n, seed)
    rng = np.random.default_rng(seed + 1)
    th[:, 0] = center[0] + width * rng.random(n)
    th[:, 1] = center[1] + width * rng.random(n)
    return th


# every (l, m) with 2 <= l <= 5: 32 modes, the widest operand (kp = 64)
LM32 = [(l, m) for l in range(2, 6) for m in range(-l, l + 1)]

SHAPES = [
    # detectors, modes (count or (l, m) list; kp = 16 ceil(2M / 16)), sampling rate, time bins
    (("H1",), 21, 8192.0, 601),                   # K = 1, kp = 48
    (("H1", "L1"), LM32, 4096.0, 257),            # K = 2, kp = 64
    (("H1", "L1", "V1", "X1"), 9, 4096.0, 401),   # K = 4, kp = 32
    (("H1", "L1", "V1", "X1"), 4, 4096.0, 129),   # K = 4, kp = 16
]


def shape_problem(i, seed):
    dets, modes, fs, n_t = SHAPES[i]
    if isinstance(modes, int):
        return S.make_problem(det_names=dets, n_modes=modes, fs=fs, n_t=n_t, seed=seed)
    return S.make_problem(det_names=dets, lm=modes, fs=fs, n_t=n_t, seed=seed)


@pytest.mark.parametrize("shape", range(len(SHAPES)))
def test_tc_kernel_shapes_match_oracle(G, orc, monkeypatch, shape):
    p = shape_problem(shape, 900 + shape)
    th = clustered(1500, 910 + shape)
    exp, _, quad = orc.lnL(p, th, want_bins=True)
    got = {}
    for tc in ("1", "0"):
        monkeypatch.setenv("RIFT_ILE_TC", tc)
        with G.ILE(p, precision=G.RIFT_FP32, max_samples=2048) as s:
            got[tc] = s.eval(th)
            assert s.plan()[0] == (G.RIFT_KERNEL_TENSOR if tc == "1" else G.RIFT_KERNEL_CUDA_CORE)
    for tc, g in got.items():
        d = np.abs(g - exp)
        assert np.max(d) <= FP32_TOL, (tc, np.max(d))


def test_tc_kernel_four_detectors_adapt_matches_fp64_path(G, monkeypatch):
    """Two adaptive iterations of a four-detector problem on the tensor-core kernel:
    ln Z of each iteration against the float64 path of the device on the same sample
    stream (the sampler draws in float64, so both paths see the same samples until the
    float32 weights move the histograms)."""
    monkeypatch.setenv("RIFT_ILE_TC", "1")
    p = S.make_problem(det_names=("H1", "L1", "V1", "X1"), n_modes=9, fs=4096.0, n_t=401, seed=931)
    n = 20000
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=n, n_bins=32, seed=5) as s:
        r32 = s.marginalize(n)
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=n, n_bins=32, seed=5) as s:
        r64 = s.marginalize(n)
    assert abs(r32["lnZ"] - r64["lnZ"]) <= 1e-3
