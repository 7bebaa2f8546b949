"""Gaussian-mixture (GMM) sampling prior of arXiv:2505.11655 Sec. II B ("the other
implementation uses Gaussian mixture models to generate sampling priors") as a plain
oracle, on the unit cube of prior-CDF coordinates v where the prior is uniform.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper names the GMM integrator but gives no algorithm; the readings here:
* C components with weights pi_c and diagonal covariances: per dimension a normal with
  mean mu_cd in [0, 1] and width sig_cd, truncated to [0, 1] so that the density has a
  closed-form normalisation:
      g(v) = sum_c pi_c prod_d phi((v_d - mu_cd)/sig_cd) / (sig_cd (Phi(b_cd) - Phi(a_cd))),
      a = -mu/sig, b = (1 - mu)/sig;
* draws: the component, then every dimension by the inverse CDF of its truncated normal
  (``orc_gmm_draw``: Philox counter words 8..11);
* initial state: pi = 1/C, sig = 0.25, means on a Kronecker lattice
  mu_cd = frac((c + 1/2) alpha_d), alpha_d = the fractional parts of sqrt(p_d) for the
  first six primes p_d (deterministic and spread over the cube);
* training: one weighted EM step per batch on every sample it is given, weights
  omega_i = exp(ln w_i - max ln w): responsibilities r_ic proportional to
  pi_c g_c(v_i); pi_c <- (1 - eps) S_c / S + eps / C, mu_cd <- sum omega r v / S_c,
  sig_cd^2 <- sum omega r (v - mu)^2 / S_c (from the first two moments), with
  S_c = sum_i omega_i r_ic; sig floored at sig_min and capped at 1, mu clipped to [0, 1];
  a component with S_c below 1e-300 S keeps its means and widths.
"""
from __future__ import annotations

import math

import numpy as np

from . import _p, lib

PRIMES = (2, 3, 5, 7, 11, 13)
SIG_INIT = 0.25


def kronecker_means(C):
    alpha = np.array([math.sqrt(p) % 1.0 for p in PRIMES])
    return np.mod((np.arange(C)[:, None] + 0.5) * alpha[None, :], 1.0)


def _phi_cdf(x):
    from scipy.special import ndtr
    return ndtr(x)


class GMM:
    """State of the Gaussian-mixture sampling prior."""

    def __init__(self, n_comp=4, seed=1, sig_min=1e-3, eps=0.02, d_min=100.0, d_max=1000.0):
        self.C = int(n_comp)
        self.seed = int(seed)
        self.sig_min = float(sig_min)
        self.eps = float(eps)
        self.d_min, self.d_max = float(d_min), float(d_max)
        self.pi = np.full(self.C, 1.0 / self.C)
        self.mu = kronecker_means(self.C)
        self.sig = np.full((self.C, 6), SIG_INIT)

    def draw(self, n, it):
        th = np.empty((n, 6))
        v = np.empty((n, 6))
        comp = np.empty(n, np.int32)
        pi, mu, sig = (np.ascontiguousarray(x, np.float64) for x in (self.pi, self.mu, self.sig))
        lib().orc_gmm_draw(_p(pi), _p(mu), _p(sig), self.C, self.seed, it, n, self.d_min, self.d_max, _p(th),
                           _p(v), _p(comp))
        return th, v, comp

    def ln_components(self, v):
        """ln(pi_c g_c(v)) [n][C] (pi normalised)."""
        v = np.asarray(v, np.float64)
        pi = self.pi / self.pi.sum()
        a, b = -self.mu / self.sig, (1.0 - self.mu) / self.sig
        lnZ = np.log(self.sig) + np.log(_phi_cdf(b) - _phi_cdf(a)) + 0.5 * math.log(2.0 * math.pi)   # [C][6]
        z = (v[:, None, :] - self.mu[None, :, :]) / self.sig[None, :, :]
        return np.log(pi)[None, :] + np.sum(-0.5 * z * z - lnZ[None, :, :], axis=2)

    def ln_density(self, v):
        lc = self.ln_components(v)
        m = lc.max(axis=1)
        return m + np.log(np.exp(lc - m[:, None]).sum(axis=1))

    def em_update(self, v, lnw):
        """One weighted EM step on samples v [n][6] with log-weights lnw [n]."""
        v = np.asarray(v, np.float64)
        lnw = np.asarray(lnw, np.float64)
        ok = np.isfinite(lnw)
        if not ok.any():
            return
        om = np.where(ok, np.exp(np.where(ok, lnw, 0.0) - lnw[ok].max()), 0.0)
        lc = self.ln_components(v)
        lc = lc - lc.max(axis=1, keepdims=True)
        r = np.exp(lc)
        r /= r.sum(axis=1, keepdims=True)
        wr = om[:, None] * r                                  # [n][C]
        S_c = wr.sum(axis=0)
        S = S_c.sum()
        m1 = wr.T @ v                                         # [C][6]
        m2 = wr.T @ (v * v)
        live = S_c > 1e-300 * S
        mu = np.where(live[:, None], m1 / np.where(live, S_c, 1.0)[:, None], self.mu)
        var = np.where(live[:, None], m2 / np.where(live, S_c, 1.0)[:, None] - mu * mu, self.sig ** 2)
        self.mu = np.clip(mu, 0.0, 1.0)
        self.sig = np.clip(np.sqrt(np.maximum(var, 0.0)), self.sig_min, 1.0)
        self.pi = (1.0 - self.eps) * S_c / S + self.eps / self.C
