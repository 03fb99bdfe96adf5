"""Eigenvalue statements of the paper as numbers, for the oracle's pins.

* Theorem 1: intervals containing eig(P_D^{-1} A) in terms of
  lambda_Phi = min(lambda_D, lambda_R), Lambda_Phi = max(Lambda_D, Lambda_R),
  lambda_S, Lambda_S, lambda_L, Lambda_L and kappa(D).
* The general block-diagonal result it rests on (Eq. BDPrecBounds) with
  delta, Delta = extreme eig(Phi_hat^{-1} Phi), phi, Phi = extreme
  eig(S_hat^{-1} S).
* Remark 1: MINRES residual bound after 2l iterations for eigenvalues in
  [-mu1, -mu2] U [mu3, mu4] with mu1 - mu2 = mu4 - mu3.
* Proposition 1: at least r s unit eigenvalues of L_M^{-T} L^T L L_M^{-1},
  r = N + 1 - 2 floor(N/k), for 2 <= k <= N+1.
* Proposition 2 / Remark 3: if ||M_i M_i^T||_2 <= 1 the eigenvalues of that
  matrix are at most k + 1 + 2 sqrt(k), tightened to 1 + k + sqrt(k) when
  floor(N/k) = 1.
"""
from __future__ import annotations

import math

import numpy as np


def bd_intervals(delta, Delta, phi, Phi):
    """Eq. BDPrecBounds: three intervals (negative, middle, positive)."""
    neg = ((delta - math.sqrt(delta ** 2 + 4 * Delta * Phi)) / 2,
           (Delta - math.sqrt(Delta ** 2 + 4 * delta * phi)) / 2)
    mid = (delta, Delta)
    pos = ((delta + math.sqrt(delta ** 2 + 4 * delta * phi)) / 2,
           (Delta + math.sqrt(Delta ** 2 + 4 * Delta * Phi)) / 2)
    return neg, mid, pos


def theorem1_intervals(lam_D, Lam_D, lam_R, Lam_R, lam_S, Lam_S, lam_L, Lam_L, kappa_D):
    lam_Phi = min(lam_D, lam_R)
    Lam_Phi = max(Lam_D, Lam_R)
    phi = lam_S * lam_L / kappa_D
    Phi = Lam_S * Lam_L * kappa_D
    return bd_intervals(lam_Phi, Lam_Phi, phi, Phi)


def in_intervals(vals, intervals, rtol=1e-9):
    ok = np.zeros(len(vals), dtype=bool)
    for lo, hi in intervals:
        pad = rtol * max(abs(lo), abs(hi), 1.0)
        ok |= (vals >= lo - pad) & (vals <= hi + pad)
    return ok


def remark1_factor(mu1, mu2, mu3, mu4):
    """Stretch the intervals so that mu1 - mu2 = mu4 - mu3, then return the
    contraction factor per two MINRES iterations."""
    w = max(mu1 - mu2, mu4 - mu3)
    if mu1 - mu2 < w:
        mu1 = mu2 + w
    else:
        mu4 = mu3 + w
    a = math.sqrt(mu1 * mu4)
    b = math.sqrt(mu2 * mu3)
    return (a - b) / (a + b)


def remark1_iterations(mu1, mu2, mu3, mu4, tol):
    """Smallest even iteration count 2l with 2 rho^l <= tol."""
    rho = remark1_factor(mu1, mu2, mu3, mu4)
    if rho <= 0:
        return 2
    l = math.ceil(math.log(tol / 2.0) / math.log(rho))
    return 2 * max(l, 1)


def prop1_unit_count(N, k, s):
    return (N + 1 - 2 * (N // k)) * s


def prop2_upper(N, k):
    if N // k == 1:
        return 1 + k + math.sqrt(k)
    return k + 1 + 2 * math.sqrt(k)
