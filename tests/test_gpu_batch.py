"""Captured adaptive sequences and batches of uneven solves.

* A replayed graph (rift_ile_adapt of a repeated shape) gives the results of direct
  launches, call after call.
* rift_batch_run over uneven solves gives what rift_ile_adapt gives on each handle
  alone, run after run, and each solve's last batch meets the oracle.
* The launch plan the autotuner picks is reported, and forced plans are honoured.

Both paths are bitwise reproducible for a fixed seed (the sampler histogram is
summed exactly, the sky sort is stable), so results are compared exactly.
"""
import os

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


def uneven_points(count=6):
    """Points of the batched workload's generator with their sample budgets scaled
    down (so that the oracle check stays quick), in uneven sizes."""
    out = []
    for i in range(count):
        p, n = S.batched_problem(i)
        out.append((p, max(600, n // 40)))
    return out


def assert_same(a, b, precision):
    for k in ("lnZ", "n_eff", "n_ess", "lnL_max", "n_total"):
        assert a[k] == b[k], (precision, k, a[k], b[k])
    assert a["lnZ_iter"] == b["lnZ_iter"]


def assert_close_arrays(x, y, precision):
    assert np.array_equal(x, y), precision


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_graph_replay_equals_direct(G, monkeypatch, precision):
    prec = G.RIFT_FP64 if precision == "fp64" else G.RIFT_FP32
    p = S.plain_fp64_problem() if precision == "fp64" else S.single_large_problem()
    n = 6000
    runs = {}
    for graphs in ("0", "1"):
        monkeypatch.setenv("RIFT_ILE_GRAPHS", graphs)
        with G.ILE(p, precision=prec, max_samples=n, n_bins=32, seed=11) as s:
            res = [s.adapt(2, n) for _ in range(4)]   # calls 2.. replay the captured graph
            th = s.last_batch(n)
            runs[graphs] = (res, th, s.sampler(), s.plan())
    (ra, tha, Pa, pa), (rb, thb, Pb, pb) = runs["0"], runs["1"]
    assert pa == pb
    for a, b in zip(ra, rb):
        assert_same(a, b, precision)
    for x, y in zip(tha[:3], thb[:3]):   # theta, ln p - ln p_s, ln L
        assert_close_arrays(x, y, precision)
    assert_close_arrays(Pa, Pb, precision)
    # the replayed calls still time their stages
    assert rb[-1]["time_ms"][3] > 0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_equals_individual_solves(G, orc, precision):
    prec = G.RIFT_FP64 if precision == "fp64" else G.RIFT_FP32
    pts = uneven_points()
    iters = [1 + i % 3 for i in range(len(pts))]
    # individually
    alone = []
    for i, (p, n) in enumerate(pts):
        with G.ILE(p, precision=prec, max_samples=n, n_bins=32, seed=21 + i) as s:
            alone.append([s.adapt(iters[i], n) for _ in range(2)] + [s.last_batch(n)])
    # as one batch, run twice
    solves = [G.ILE(p, precision=prec, max_samples=n, n_bins=32, seed=21 + i) for i, (p, n) in enumerate(pts)]
    try:
        with G.Batch(solves, iters, [n for _, n in pts]) as b:
            first, rc1 = b.run()
            second, rc2 = b.run()
            assert rc1 == 0 and rc2 == 0
            assert b.kernel_launches() > 10 * len(pts)
        last = [s.last_batch(n) for s, (_, n) in zip(solves, pts)]
    finally:
        for s in solves:
            s.close()
    for i, (p, n) in enumerate(pts):
        for got, exp in ((first[i], alone[i][0]), (second[i], alone[i][1])):
            assert got["status"] == 0
            assert_same(got, exp, precision)
            assert got["n_total"] == iters[i] * n
        for x, y in zip(last[i][:3], alone[i][2][:3]):
            assert_close_arrays(x, y, precision)
    # each solve's last batch against the oracle on the device's own samples
    for i, (p, n) in enumerate(pts):
        th, lr, ll, lw = last[i]
        red = orc.reduce(orc.lnL(p, th) + lr)
        tol = 1e-9 * max(1.0, abs(red["lnZ"])) if precision == "fp64" else 1e-3
        assert abs(second[i]["lnZ_iter"][-1] - red["lnZ"]) <= tol, (i, second[i]["lnZ_iter"][-1], red["lnZ"])


def test_plans_reported_and_forced(G, monkeypatch):
    p = S.single_large_problem()
    n = 5000
    with G.ILE(p, precision=G.RIFT_FP64, max_samples=n) as s:
        s.adapt(1, n)
        assert s.plan()[0] == G.RIFT_KERNEL_FP64
    for env, kern in (("1", G.RIFT_KERNEL_TENSOR), ("0", G.RIFT_KERNEL_CUDA_CORE)):
        monkeypatch.setenv("RIFT_ILE_TC", env)
        with G.ILE(p, precision=G.RIFT_FP32, max_samples=n) as s:
            s.adapt(1, n)
            assert s.plan() == (kern, 4)
    monkeypatch.delenv("RIFT_ILE_TC")
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=n) as s:
        s.adapt(1, n)
        k, cell = s.plan()
        assert k in (G.RIFT_KERNEL_TENSOR, G.RIFT_KERNEL_CUDA_CORE) and cell in (2, 4, 8)


def test_tuner_appends_new_classes_to_cache_file(G, monkeypatch, tmp_path):
    path = tmp_path / "plans.txt"
    monkeypatch.setenv("RIFT_ILE_TUNE_CACHE", str(path))
    # a class no other test uses: one detector, 5 modes, 333 bins
    p = S.make_problem(("L1",), 5, 4096.0, n_t=333, snr=15.0, seed=S.config_seed(3, 9001))
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=9000) as s:
        s.adapt(1, 9000)
        k, cell = s.plan()
    lines = path.read_text().split()
    assert len(lines) == 4 and lines[0].startswith("K1_kp1_nt333_")
    assert int(lines[1]) == (1 if k == G.RIFT_KERNEL_TENSOR else 0) and int(lines[2]) == cell
    assert lines[3] == "0"   # the three-delay key is a candidate only with three detectors


def test_tuner_adapted_class(G, monkeypatch, tmp_path):
    """A sampler adapted twice, on a batch of 2^19 samples or more, re-times the
    tensor-core plans once for its class (a second cache line, "_adapted"); smaller
    batches keep their first plan."""
    path = tmp_path / "plans.txt"
    monkeypatch.setenv("RIFT_ILE_TUNE_CACHE", str(path))
    p = S.make_problem(("H1", "L1", "V1"), 7, 4096.0, n_t=301, snr=20.0, seed=S.config_seed(3, 9002))
    n = 1 << 19
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=n) as s:
        plans = []
        for _ in range(4):
            r = s.adapt(1, n)
            assert r["status"] == 0
            plans.append(s.plan())
    lines = [ln.split() for ln in path.read_text().splitlines()]
    keys = [ln[0] for ln in lines]
    assert len(lines) == 2 and keys[1] == keys[0] + "_adapted", lines
    if int(lines[0][1]) == 1:
        assert int(lines[1][1]) == 1   # the kernel family stays
    else:
        assert lines[1][1:] == lines[0][1:]
    assert plans[0] == plans[1]   # iterations 0 and 1: the first plan
    with G.ILE(p, precision=G.RIFT_FP32, max_samples=n // 4) as s:
        for _ in range(3):
            s.adapt(1, n // 4)
    assert len(path.read_text().splitlines()) == 3   # its own first class only, no adapted class


@pytest.mark.slow
def test_batched_workload_every_point_meets_oracle(G, orc):
    """All 512 points of the batched uneven workload (sizes, detectors, modes, rates and
    bin counts as the benchmark draws them; sample budgets capped at 2000 so that the
    oracle check stays quick) as one float32 batch: every point's last-iteration ln Z
    is within 1e-3 of the oracle's float64 reduction of that point's own last batch."""
    pts = []
    for i in range(512):
        p, n = S.batched_problem(i)
        pts.append((p, max(300, min(2000, n // 40))))
    iters = [1 + i % 3 for i in range(len(pts))]
    solves = [G.ILE(p, precision=G.RIFT_FP32, max_samples=n, n_bins=32, seed=41 + i) for i, (p, n) in enumerate(pts)]
    try:
        with G.Batch(solves, iters, [n for _, n in pts]) as b:
            res, rc = b.run()
            assert rc == 0
        last = [s.last_batch(n) for s, (_, n) in zip(solves, pts)]
    finally:
        for s in solves:
            s.close()
    worst = 0.0
    for i, (p, n) in enumerate(pts):
        assert res[i]["status"] == 0 and res[i]["n_total"] == iters[i] * n
        th, lr, ll, lw = last[i]
        red = orc.reduce(orc.lnL(p, th) + lr)
        d = abs(res[i]["lnZ_iter"][-1] - red["lnZ"])
        worst = max(worst, d)
        assert d <= 1e-3, (i, res[i]["lnZ_iter"][-1], red["lnZ"])
    print("max |d lnZ| over 512 points:", worst)
