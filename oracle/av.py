"""Adaptive-volume (AV) integrator of arXiv:2505.11655, Sec. IV A, as a plain
step-by-step oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The integrator works on the unit cube of prior-CDF coordinates v in [0,1)^6 (the
prior is uniform there, so the evidence is Z = int L dv).  Each iteration g:

1. draw n points uniformly over the union of the active cells (grid of 2^level cells
   per side; the draw itself is ``orc_av_draw``); sampling density 1/V_g with V_g the
   cells' total volume, so ln w = ln L + ln V_g;
2. evaluate ln L (any callable: the ILE likelihood, or an analytic target in the pins);
3. add to the live set the fresh points that pass the current threshold, in index
   order and while the live set has room;
4. threshold: histogram the live ln L in bins of 1/64 below the live maximum m (4096
   bins; bin b = floor((m - ln L) 64)) with exact fixed-point masses
   floor(exp(ln L - m) 2^S), S = 62 - ceil(log2 N_live), and counts; the kept bins are
   the fewest from the top that hold both the fraction P_thr of the mass
   (floor(P_thr 2^20) / 2^20, compared exactly) and at least N_min* points: N_min* is a
   floor (while the likelihood is poorly resolved a handful of points carry P_thr of the
   mass and the top N_min* points set the threshold; once the mass is spread over more
   points, the P_thr rule does); N_min = the points kept;
5. refine: V' = V_g N_min / N_live, dV = V' / sqrt(N_min), n_bins = (1/dV)^(1/6);
   the new level is floor(log2 n_bins), at least the current one and at most 10, so
   that a cell holds of order sqrt(N_min) points (Eq. nbins_V: cells no smaller than the
   volume's sampling uncertainty); the new active cells are those holding a kept live
   point, and the live set is cut to the kept points.

Readings where the paper is silent: the histogram threshold (bin width 1/64), the
fixed-point mass comparison, power-of-two nested grids (so that refined cells lie
inside active ones), rounding n_bins down, and the estimator: every iteration's fresh
draws are weighted by their own V_g and pooled, as for the histogram sampler.
"""
from __future__ import annotations

import math

import numpy as np

from . import _p, lib, reduce

LN_BINS_PER_UNIT = 64
N_HIST = 4096
P_SHIFT = 20
MAX_LEVEL = 10


def cell_keys(v, level):
    """Packed integer coordinates of the cells (2^level per side) holding points v [n][6]."""
    c = np.floor(np.asarray(v) * float(1 << level)).astype(np.uint64)
    key = np.zeros(c.shape[0], np.uint64)
    for d in range(6):
        key |= c[:, d] << np.uint64(level * d)
    return key


def fix_shift(n):
    return 62 - max(0, math.ceil(math.log2(max(1, n))))


def threshold(lnL, p_thr, n_min_star):
    """(m, b_thr, kept mask) of the live ln L under the histogram rule (step 4)."""
    lnL = np.asarray(lnL, np.float64)
    m = float(np.max(lnL))
    b = np.floor((m - lnL) * LN_BINS_PER_UNIT)
    valid = b < N_HIST
    bi = b[valid].astype(np.int64)
    S = fix_shift(lnL.size)
    mass = [0] * N_HIST
    count = [0] * N_HIST
    for x, k in zip(lnL[valid], bi):
        mass[k] += int(math.ldexp(math.exp(x - m), S))
        count[k] += 1
    total = sum(mass)
    p_num = int(math.floor(p_thr * (1 << P_SHIFT)))
    need = min(n_min_star, lnL.size)
    run_m = run_c = 0
    b_mass = b_count = None
    for k in range(N_HIST):
        run_m += mass[k]
        run_c += count[k]
        if b_mass is None and (run_m << P_SHIFT) >= p_num * total:
            b_mass = k
        if b_count is None and run_c >= need:
            b_count = k
        if b_mass is not None and b_count is not None:
            break
    # N_min* is a floor: while a few points carry P_thr of the mass (a poorly resolved
    # likelihood) the top N_min* points are kept; once the mass is spread over more
    # points the P_thr rule keeps them
    if b_count is None:
        # the N_min*-th largest value lies beyond the histogram's range: its bin, exactly
        b_count = int(np.floor((m - np.sort(lnL)[::-1][need - 1]) * LN_BINS_PER_UNIT))
    b_thr = max(b_mass if b_mass is not None else N_HIST - 1, b_count)
    kept = b <= b_thr
    return m, b_thr, kept


def next_level(level, V, n_min, n_live):
    v_next = V * n_min / n_live
    dV = v_next / math.sqrt(n_min)
    nb = (1.0 / dV) ** (1.0 / 6.0)
    cand = int(math.floor(math.log2(nb))) if nb >= 1.0 else 0
    return max(level, min(MAX_LEVEL, cand))


class AV:
    """State of the adaptive-volume integrator."""

    def __init__(self, seed=1, p_thr=0.9999, n_min_star=1000, capacity=1 << 22, d_min=100.0, d_max=1000.0):
        self.seed = int(seed)
        self.p_thr = float(p_thr)
        self.n_min_star = int(n_min_star)
        self.capacity = int(capacity)
        self.d_min, self.d_max = float(d_min), float(d_max)
        self.level = 0
        self.cells = np.zeros(1, np.uint64)
        self.V = 1.0        # volume of the active cells (the sampling density is 1/V)
        self.V_thr = 1.0    # estimated volume above the current threshold (V_g of Eq. nbins_V)
        self.live_v = np.zeros((0, 6))
        self.live_lnL = np.zeros(0)
        self.thr = None   # (m, b) of the previous threshold
        self.iteration = 0

    def draw(self, n, it=None):
        it = self.iteration if it is None else it
        th = np.empty((n, 6))
        v = np.empty((n, 6))
        cells = np.ascontiguousarray(self.cells, np.uint64)
        lib().orc_av_draw(_p(cells), cells.size, self.level, self.seed, it, 0, n, self.d_min, self.d_max,
                          _p(th), _p(v))
        return th, v

    def step(self, lnL_fn, n):
        """One iteration; returns dict(theta, v, lnL, lnw, level, n_cells, V, n_live, n_min)."""
        V_draw, level_draw, ncell_draw = self.V, self.level, self.cells.size
        th, v = self.draw(n)
        ll = np.asarray(lnL_fn(th), np.float64)
        lnw = ll + math.log(V_draw)
        rec = self.update(v, ll)
        rec.update(theta=th, v=v, lnL=ll, lnw=lnw, level=level_draw, n_cells=ncell_draw, V=V_draw)
        return rec

    def contains(self, v):
        """Whether points v [n][6] lie in the active cells."""
        keys = cell_keys(v, self.level)
        pos = np.searchsorted(self.cells, keys)
        return (pos < self.cells.size) & (self.cells[np.minimum(pos, self.cells.size - 1)] == keys)

    def update(self, v, ll):
        """Steps 3-5 on fresh points v [n][6] with ln L values ll (index order); returns
        dict(n_live, n_min, next_level, next_cells)."""
        n = ll.size
        # 3. live set
        if self.thr is None:
            keep = np.ones(n, bool)
        else:
            m0, b0 = self.thr
            keep = np.floor((m0 - ll) * LN_BINS_PER_UNIT) <= b0
        room = self.capacity - self.live_lnL.size
        idx = np.nonzero(keep)[0][:max(0, room)]
        self.live_v = np.concatenate([self.live_v, v[idx]])
        self.live_lnL = np.concatenate([self.live_lnL, ll[idx]])
        n_live = self.live_lnL.size
        # 4. threshold
        m, b_thr, kept = threshold(self.live_lnL, self.p_thr, self.n_min_star)
        n_min = int(kept.sum())
        # 5. refine
        self.level = next_level(self.level, self.V_thr, n_min, n_live)
        self.V_thr = self.V_thr * n_min / n_live
        self.live_v = self.live_v[kept]
        self.live_lnL = self.live_lnL[kept]
        self.cells = np.unique(cell_keys(self.live_v, self.level))
        self.V = self.cells.size * 2.0 ** (-6 * self.level)
        self.thr = (m, b_thr)
        self.iteration += 1
        return dict(n_live=n_live, n_min=n_min, next_level=self.level, next_cells=self.cells.size)


def run(lnL_fn, n_iter, n, **kw):
    """n_iter AV iterations of n draws: per-iteration records, pooled ln Z."""
    av = AV(**kw)
    its = [av.step(lnL_fn, n) for _ in range(n_iter)]
    pooled = reduce(np.concatenate([r["lnw"] for r in its]))
    for r in its:
        r["reduce"] = reduce(r["lnw"])
    return dict(iterations=its, pooled=pooled, av=av)
