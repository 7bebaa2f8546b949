"""Overlaps Q, U, V from frequency-domain inputs (arXiv:2505.11655, Sec. II A, Eq. QUV),
as a plain oracle.  TEST INFRASTRUCTURE ONLY (see the package docstring).

On a discrete two-sided frequency grid f_j (mirror symmetric: f_{F-1-j} = -f_j) with
inverse-PSD weights w_k(f), mode waveforms h_lm(f) (shared by the detectors) and data
d_k(f):

    Q_k,lm(t)    = 2 sum_j w_k(f_j) exp(2 pi i f_j t) conj(h_lm(f_j)) d_k(f_j)
    U_k,lm,l'm'  = 2 sum_j w_k(f_j) conj(h_lm(f_j)) h_l'm'(f_j)
    V_k,lm,l'm'  = 2 sum_j w_k(f_j) h_lm(-f_j) h_l'm'(f_j)

Q is evaluated on each detector's Q grid t_s = q_t0_k + s / f_s, s = 0 .. n_q - 1.
Every sum is written out over the whole grid (no Hermitian halving, no FFT).
"""
from __future__ import annotations

import math

import numpy as np


def overlaps(freqs, h, data, w, q_t0, fs, n_q):
    """(Q [K][M][n_q], U [K][M][M], V [K][M][M]) complex128."""
    f = np.asarray(freqs, np.float64)
    h = np.asarray(h, np.complex128)
    d = np.asarray(data, np.complex128)
    w = np.asarray(w, np.float64)
    K, M, F = d.shape[0], h.shape[0], f.size
    mirror = np.arange(F)[::-1]
    Q = np.zeros((K, M, n_q), np.complex128)
    U = np.zeros((K, M, M), np.complex128)
    V = np.zeros((K, M, M), np.complex128)
    for k in range(K):
        t = q_t0[k] + np.arange(n_q) / fs
        phase = np.exp(2j * math.pi * np.outer(t, f))              # [n_q][F]
        for m in range(M):
            Q[k, m] = 2.0 * phase @ (w[k] * np.conj(h[m]) * d[k])
        for a in range(M):
            for b in range(M):
                U[k, a, b] = 2.0 * np.sum(w[k] * np.conj(h[a]) * h[b])
                V[k, a, b] = 2.0 * np.sum(w[k] * h[a][mirror] * h[b])
    return Q, U, V
