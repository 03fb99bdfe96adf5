"""SOAR covariances and the observation-error approximations R-hat.

Sec. 6.1 builds B and Q from a second-order auto-regressive (SOAR) correlation
(Eq. SOAR).  As printed that formula does not decay with distance (the
exponential multiplies only the distance term), so this oracle takes the
standard SOAR function it cites [Yaglom87]:

    c(r) = sigma2 * (1 + r/ell) * exp(-r/ell),

with r the chordal distance between two points of the periodic unit domain
(circle of circumference 1): r = sin(pi*|x_i - x_j|)/pi.  Chordal distance
keeps the matrix positive definite on the circle, so no diagonal shift is
added (the paper's random shift delta, Sec. 6.1, is dropped).  The same
function over the observed positions x_j = obs_idx[j]/s gives R_i.

Sec. 5.2 defines the reconditioning-based approximations:
  Alg. 1 (ridge regression)  R_RR = R + gamma I,
         gamma = (lambda_max - lambda_min kappa_max)/(kappa_max - 1), clamped at 0
         when R is already better conditioned than kappa_max;
  Alg. 2 (minimum eigenvalue) R_ME = V diag(max(lambda_k, T)) V^T,
         T = lambda_max/kappa_max; if T <= lambda_min then R_ME = R.
Sec. 5.1: R_diag = diag(R).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def chordal_distance(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Chordal distance on the circle of circumference 1 between positions in
    [0,1): |chord| = sin(pi*|x-y|)/pi."""
    d = np.abs(x[:, None] - y[None, :])
    return np.sin(np.pi * d) / np.pi


def soar_function(r: np.ndarray, sigma2: float, length: float) -> np.ndarray:
    q = r / length
    return sigma2 * (1.0 + q) * np.exp(-q)


def soar_matrix(positions: np.ndarray, sigma2: float, length: float) -> np.ndarray:
    """Dense SOAR covariance over the given positions (Sec. 6.1)."""
    r = chordal_distance(positions, positions)
    return soar_function(r, sigma2, length)


def grid_positions(s: int) -> np.ndarray:
    return np.arange(s, dtype=np.float64) / s


def soar_state(s: int, sigma2: float, length: float) -> np.ndarray:
    """B or Q on the full periodic grid: an s x s circulant matrix."""
    return soar_matrix(grid_positions(s), sigma2, length)


def soar_obs(s: int, obs_idx: np.ndarray, sigma2: float, length: float) -> np.ndarray:
    """R_i: SOAR over the observed grid positions."""
    return soar_matrix(np.asarray(obs_idx, dtype=np.float64) / s, sigma2, length)


def ridge_gamma(lam_min: float, lam_max: float, kappa_max: float) -> float:
    """Alg. 1 shift, clamped at zero (R already at or below kappa_max)."""
    g = (lam_max - lam_min * kappa_max) / (kappa_max - 1.0)
    return max(g, 0.0)


def r_ridge(R: np.ndarray, kappa_max: float):
    """Alg. 1: R_RR = R + gamma I.  Returns (R_RR, gamma)."""
    lam = np.linalg.eigvalsh(R)
    gamma = ridge_gamma(lam[0], lam[-1], kappa_max)
    return R + gamma * np.eye(R.shape[0]), gamma


def r_min_eig(R: np.ndarray, kappa_max: float):
    """Alg. 2: eigenvalues at or below T = lambda_max/kappa_max are raised to T.
    Returns (R_ME, T)."""
    lam, V = np.linalg.eigh(R)
    T = lam[-1] / kappa_max
    if T <= lam[0]:
        return R.copy(), T
    lam_me = np.where(lam > T, lam, T)
    return (V * lam_me) @ V.T, T


def r_diag(R: np.ndarray) -> np.ndarray:
    """Sec. 5.1: the diagonal of R."""
    return np.diag(np.diag(R))


def rhat(R: np.ndarray, kind: str, kappa_max: float = 100.0) -> np.ndarray:
    if kind == "exact":
        return R.copy()
    if kind == "rr":
        return r_ridge(R, kappa_max)[0]
    if kind == "me":
        return r_min_eig(R, kappa_max)[0]
    if kind == "diag":
        return r_diag(R)
    raise ValueError(kind)


class SPDSolver:
    """x = M^{-1} v through a Cholesky factorisation (the exact-Cholesky
    reading of the paper's incomplete Cholesky on dense blocks)."""

    def __init__(self, M: np.ndarray):
        self.factor = sla.cho_factor(M, lower=True)

    def __call__(self, v: np.ndarray) -> np.ndarray:
        return sla.cho_solve(self.factor, v)
