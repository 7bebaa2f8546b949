"""Portfolio integrator of arXiv:2505.11655, Sec. IV ("Portfolio integrator"), as a
plain step-by-step oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The members are the product-form histogram sampler (Sec. II B, ``oracle.Sampler``), the
adaptive-volume integrator (Sec. IV A, ``oracle.av.AV``) and the Gaussian-mixture sampling
prior (Sec. II B, ``oracle.gmm.GMM``).  All sample the unit cube of prior-CDF
coordinates v, where the prior is uniform, so each member's sampling prior is a density
g_alpha(v) relative to the prior:

  g_hist(v) = prod_d B P_d[b_d] / sum_b P_d[b]   (b_d the histogram bin of v_d)
  g_AV(v)   = 1/V on the active cells, 0 elsewhere
  g_GMM(v)  = the truncated mixture density.

The portfolio's sampling prior is the weighted average p_s/p = sum_alpha W_alpha g_alpha
with sum_alpha W_alpha = 1 over the active members.  One iteration g:

1. member choice: with x = U_i 2^-53 from ``orc_portfolio_members`` (Philox counter
   (i, g, 7)), draw i comes from the histogram when x < W_hist, from the AV member when
   x < W_hist + W_AV, else from the GMM; each member's draws use its own counters of
   iteration g (``orc_draw``, ``orc_av_draw``, ``orc_gmm_draw``);
2. ln w = ln L - ln(sum_alpha W_alpha g_alpha(v)): the histogram bin of another member's
   draw is floor(v_d B), an AV cell holds a draw when its key at the current level is
   active.  With a single active member ln w is that member's own ln L + ln(p/p_s);
3. weights: per member, the effective sample size n_ESS,alpha = (sum w)^2 / sum w^2 over
   the batch's draws from that member (the overall weights w above); W' proportional to
   n_ESS; then no weight below 0.05/N_s (N_s the number of active members): those below
   are set to the floor and the others scaled to fill the rest, repeated until none is
   below.  With adaptation off the weights stay as given;
4. training: a member whose new weight is below 0.05 is frozen (not trained).  The
   histogram and the GMM train on every sample of the batch with the overall ln w
   (``orc_adapt``; one weighted EM step); the AV member on its own draws (v, ln L) in index
   order (its live set, threshold and refinement count live points among uniform draws
   over its own active cells, which only its own draws are).  A member that drew nothing
   is not trained (the AV member) or trains on the others' draws (histogram, GMM).

Activation: the AV and GMM members join at iterations ``av_start`` and ``gmm_start``;
before, the members active so far draw alone; when one joins, the weights are reset to the
initial ones (normalised over the active members).

Readings where the paper is silent or leaves a choice: the per-member n_ESS uses the
overall weights of that member's draws; the floor is applied by the water-filling rule
above; the freeze rule reads the new weight; the AV member learns from its own draws
(the paper allows a member not to train on the others' output); a joining member starts
from the initial weights.
"""
from __future__ import annotations

import math

import numpy as np

from . import Sampler, _p, lib, reduce
from .av import AV
from .gmm import GMM

HIST, AVM, GMMM = 0, 1, 2
W_FLOOR = 0.05      # the floor is W_FLOOR / N_s
FREEZE_BELOW = 0.05


def floor_weights(W, active, floor):
    """Normalised weights with no active entry below `floor` (water-filling); inactive
    entries are 0."""
    W = np.where(active, np.asarray(W, np.float64), 0.0)
    W = W / W.sum()
    fixed = np.zeros(W.size, bool)
    while True:
        low = active & ~fixed & (W < floor)
        if not low.any():
            return W
        fixed |= low
        free = active & ~fixed
        W[fixed] = floor
        W[free] *= (1.0 - floor * fixed.sum()) / W[free].sum()


def member_ess(lnw, member, n_members=3):
    """n_ESS and draw count of each member's draws in one batch."""
    ess, cnt = np.zeros(n_members), np.zeros(n_members, np.int64)
    for a in range(n_members):
        sel = member == a
        cnt[a] = int(sel.sum())
        if cnt[a] and np.isfinite(lnw[sel]).any():
            ess[a] = reduce(lnw[sel])["n_ess"]
    return ess, cnt


def choice_thresholds(W, act):
    """(t0, t1) of the member choice for normalised weights W over active members act."""
    t0 = W[HIST]
    t1 = W[HIST] + W[AVM] if act[GMMM] else 2.0
    return t0, t1


class Portfolio:
    """State of the portfolio over (histogram sampler, AV integrator, GMM)."""

    def __init__(self, members=(True, True), av_start=0, gmm_start=0, adapt_weights=True, w_init=(0.5, 0.5),
                 seed=1, n_bins=64, floor=0.1, temper=1.0, p_thr=0.9999, n_min_star=1000, capacity=1 << 22,
                 gmm_components=4, d_min=100.0, d_max=1000.0):
        m = list(members) + [False] * (3 - len(members))
        w = list(w_init) + [0.0] * (3 - len(w_init))
        self.members = np.array(m, bool)
        self.av_start = int(av_start)
        self.gmm_start = int(gmm_start)
        self.adapt_weights = bool(adapt_weights)
        self.w_init = np.array(w, np.float64)
        self.seed = int(seed)
        self.hist = Sampler(n_bins=n_bins, seed=seed, floor=floor, temper=temper, d_min=d_min, d_max=d_max)
        self.av = AV(seed=seed, p_thr=p_thr, n_min_star=n_min_star, capacity=capacity, d_min=d_min, d_max=d_max)
        self.gmm = GMM(n_comp=gmm_components, seed=seed, d_min=d_min, d_max=d_max)
        self.iteration = 0
        self.W = None

    def active(self, g):
        return np.array([self.members[HIST], self.members[AVM] and g >= self.av_start,
                         self.members[GMMM] and g >= self.gmm_start])

    def step(self, lnL_fn, n):
        """One iteration; lnL_fn(theta [n][6], v [n][6]) -> ln L.  Returns a record."""
        g = self.iteration
        act = self.active(g)
        joins = (self.members[AVM] and self.av_start > 0 and g == self.av_start) or \
                (self.members[GMMM] and self.gmm_start > 0 and g == self.gmm_start)
        if self.W is None or joins:
            self.W = floor_weights(self.w_init, act, 0.0)
        W = self.W.copy()
        n_act = int(act.sum())
        # 1. member choice and draws
        if n_act > 1:
            member = np.empty(n, np.int32)
            t0, t1 = choice_thresholds(W, act)
            lib().orc_portfolio_members(self.seed, g, n, float(t0), float(t1), _p(member))
        else:
            member = np.full(n, int(np.argmax(act)), np.int32)
        th = np.empty((n, 6))
        v = np.empty((n, 6))
        bins = np.zeros((n, 6), np.int32)
        lr = np.empty(n)
        sel = [member == a for a in range(3)]
        if sel[HIST].any():
            th_h, lr_h, b_h, v_h = self.hist.draw(n, it=g, want_v=True)
            h = sel[HIST]
            th[h], v[h], bins[h], lr[h] = th_h[h], v_h[h], b_h[h], lr_h[h]
        if sel[AVM].any():
            th_a, v_a = self.av.draw(n, it=g)
            a = sel[AVM]
            th[a], v[a] = th_a[a], v_a[a]
            lr[a] = math.log(self.av.V)
        if sel[GMMM].any():
            th_g, v_g, _ = self.gmm.draw(n, it=g)
            q = sel[GMMM]
            th[q], v[q] = th_g[q], v_g[q]
            lr[q] = -self.gmm.ln_density(v[q])
        # 2. the mixture density
        if n_act > 1:
            dens = np.zeros(n)
            if act[HIST]:
                lnd_h, b_all = self.hist.ln_density(v)
                nh = ~sel[HIST]
                bins[nh] = b_all[nh]
                lnd_h[sel[HIST]] = -lr[sel[HIST]]   # the histogram draws' own densities and bins
                dens = dens + W[HIST] * np.exp(lnd_h)
            if act[AVM]:
                dens = dens + W[AVM] * np.where(self.av.contains(v) | sel[AVM], 1.0 / self.av.V, 0.0)
            if act[GMMM]:
                dens = dens + W[GMMM] * np.exp(self.gmm.ln_density(v))
            lr = -np.log(dens)
        ll = np.asarray(lnL_fn(th, v), np.float64)
        lnw = ll + lr
        # 3. weights
        if n_act > 1:
            ess, cnt = member_ess(lnw, member)
        else:
            ess = np.where(act, reduce(lnw)["n_ess"], 0.0)
            cnt = np.where(act, n, 0)
        W_next = W
        if self.adapt_weights and n_act > 1 and ess.sum() > 0.0:
            W_next = floor_weights(ess, act, W_FLOOR / n_act)
        # 4. training
        frozen = ~act | (W_next < FREEZE_BELOW)
        if not frozen[HIST]:
            self.hist.adapt(bins, lnw)
        if not frozen[AVM] and cnt[AVM] > 0:
            self.av.update(v[sel[AVM]], ll[sel[AVM]])
        if not frozen[GMMM]:
            self.gmm.em_update(v, lnw)
        av_state = (self.av.level, self.av.cells.size, self.av.V)
        self.W = W_next
        self.iteration += 1
        return dict(theta=th, v=v, member=member, lnL=ll, lr=lr, lnw=lnw, W=W, n_ess=ess, n_drawn=cnt,
                    W_next=W_next.copy(), frozen=frozen, av_state=av_state,
                    gmm=(self.gmm.pi.copy(), self.gmm.mu.copy(), self.gmm.sig.copy()))


def run(lnL_fn, n_iter, n, **kw):
    """n_iter portfolio iterations of n draws: per-iteration records and pooled ln Z."""
    pf = Portfolio(**kw)
    its = [pf.step(lnL_fn, n) for _ in range(n_iter)]
    pooled = reduce(np.concatenate([r["lnw"] for r in its]))
    for r in its:
        r["reduce"] = reduce(r["lnw"])
    return dict(iterations=its, pooled=pooled, portfolio=pf)
