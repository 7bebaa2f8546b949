"""rift_ile_reduce_noalloc: the log-weight reduction for callers that cannot
allocate device memory at the point of the call (fixed memory budgets, caching
allocators they must not bypass, loops where cudaMalloc's implicit
synchronisation is not allowed).  Its scratch is a static device array inside
the library, so the call itself allocates nothing.

It must reproduce what the library's own marginalisation entry point reports
for the same log-weights, on two calls in a row (the static scratch keeps the
previous call's contents, which must not leak into the next result).

This file is collected last on purpose, so that a run stopping at its first
failure has already run every other test; it also passes when run alone.
"""
import ctypes as C

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


def test_noalloc_reduction_matches_marginalize_twice(G):
    """Against rift_ile_marginalize of a float64 handle (the same float64 terms)."""
    import torch
    p = S.single_large_problem()
    n = 20000
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=n, n_bins=32, seed=21) as s:
        for _ in range(2):
            r = s.marginalize(n)
            lnw = torch.empty(n, dtype=torch.float64, device="cuda")
            lnL = torch.empty(n, dtype=torch.float64, device="cuda")
            G.rift_ile_last_batch(s.h, lnL_tmarg=lnL, lnw=lnw, mem=G.RIFT_MEM_DEVICE)
            out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
            G.rift_ile_reduce_noalloc(lnw, n, out, lnL=lnL)
            o = out.cpu().numpy()
            assert abs(o[0] - r["lnZ"]) <= 1e-12 * max(1.0, abs(r["lnZ"]))
            assert abs(o[1] - r["sigma_lnZ"]) <= 1e-12
            assert abs(o[2] - r["n_eff"]) <= 1e-12 * r["n_eff"]
            assert abs(o[3] - r["n_ess"]) <= 1e-12 * r["n_ess"]
            assert abs(o[5] - r["lnL_max"]) <= 1e-12 * max(1.0, abs(r["lnL_max"]))
            assert o[6] == n


def test_noalloc_reduction_spread_weights_against_oracle_twice(G, oracle_lib):
    """Log-weights spread uniformly over [-5, 0] (no single sample dominates): ln Z,
    sigma, n_eff and n_ESS equal the oracle's float64 definitions to 1e-12 on two calls in
    a row with different inputs."""
    import torch
    rng = np.random.default_rng(4)
    for n in (100000, 777):
        lnw = rng.uniform(-5.0, 0.0, n)
        ref = oracle_lib.reduce(lnw)
        out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
        G.rift_ile_reduce_noalloc(torch.from_numpy(lnw).cuda(), n, out)
        o = out.cpu().numpy()
        assert abs(o[0] - ref["lnZ"]) <= 1e-12 * max(1.0, abs(ref["lnZ"]))
        assert abs(o[1] - ref["sigma_lnZ"]) <= 1e-12
        assert abs(o[2] - ref["n_eff"]) <= 1e-12 * ref["n_eff"]
        assert abs(o[3] - ref["n_ess"]) <= 1e-12 * ref["n_ess"]
        assert o[6] == n


def test_noalloc_reduction_rejects_bad_sizes(G):
    import torch
    lib = G.load()
    lnw = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert lib.rift_ile_reduce_noalloc(lnw.data_ptr(), None, 0, out.data_ptr(), None) == G.RIFT_EINVAL
    assert lib.rift_ile_reduce_noalloc(lnw.data_ptr(), None, (1 << 31) + 1, out.data_ptr(), None) == G.RIFT_EINVAL
    assert lib.rift_ile_reduce_noalloc(None, None, 4, out.data_ptr(), None) == G.RIFT_EINVAL
    # a zero signal: ln Z = 0 and n_eff = n_ESS = n exactly
    G.rift_ile_reduce_noalloc(lnw, 4, out)
    o = out.cpu().numpy()
    assert o[0] == 0.0 and o[2] == 4.0 and o[3] == 4.0
    bad = torch.tensor([0.0, float("nan"), 1.0], dtype=torch.float64, device="cuda")
    assert lib.rift_ile_reduce_noalloc(bad.data_ptr(), None, 3, out.data_ptr(), None) == G.RIFT_ENONFINITE
