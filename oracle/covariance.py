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
Sec. 5.1: R_diag = diag(R); R_block (Alg. 3) keeps R's entries inside runs of
channel blocks whose first super-diagonal coupling has a scaled Frobenius
norm of at least ``tol`` and zeros the coupling between runs.

The heat-equation experiments (Sec. 6.1, Sec. 7.2) build B and Q from the
banded "modified SOAR" instead: a symmetric circulant matrix whose first row
carries amp (1 + d_i/L) exp(-d_i/L) at offsets |i| <= maxval, with
d_i = 2 |sin(i theta / 2)| and theta = pi / maxval, and zeros elsewhere (the
number of non-zeros per row does not grow with s).  Read as the standard SOAR
shape (the printed formula does not decay, as above) over that chord
distance, with the support |i| <= maxval (the half circle theta spans).  When
the banded matrix has a negative eigenvalue, |lambda_min| + psi is added to its
diagonal, psi a draw in [0, 0.5].  The channel-block R_i of Sec. 6.1: U holds,
for each channel block, the Hadamard product of a sparse random matrix and a
modified SOAR block and, above the diagonal, sparse random blocks with entries
in (0, pcorr) for each pair of channel blocks; R_i = U + U^T, shifted so that
its smallest eigenvalue is exactly 0.41 (the value Table 2 fixes).
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


# ------------------------------------------------------ R_block (Alg. 3)
def block_starts(pvec) -> np.ndarray:
    """pst of Alg. 3 (0-based, with the end p appended): block k spans rows
    pst[k] .. pst[k+1]-1."""
    return np.concatenate([[0], np.cumsum(np.asarray(pvec, dtype=np.int64))])


def block_normvec(R: np.ndarray, pvec) -> np.ndarray:
    """Alg. 3: Frobenius norm of each first super-diagonal block (j, j+1),
    divided by sqrt(pvec_j pvec_{j+1})."""
    pst = block_starts(pvec)
    out = np.zeros(len(pvec) - 1)
    for j in range(len(pvec) - 1):
        blk = R[pst[j]:pst[j + 1], pst[j + 1]:pst[j + 2]]
        out[j] = np.sqrt(np.sum(blk * blk)) / np.sqrt(float(pvec[j]) * float(pvec[j + 1]))
    return out


def _runs(cuts, p):
    b = [0] + sorted(cuts) + [p]
    return [(b[i], b[i + 1]) for i in range(len(b) - 1)]


def r_block_cuts(R: np.ndarray, pvec, tol: float, maxsize=None, numproc=None):
    """The rows at which Alg. 3 decouples R: R_block couples rows a < b only
    when no cut c has a < c <= b.  Readings: a "block" of the size and count
    rules is a run of channel blocks between cuts; splitting a run cuts it at
    its row midpoint (floor), first run on ties, runs of one row are not split;
    combining joins the adjacent pair of runs with the smallest total size
    (first on ties); each rule is applied once, in the printed order.  Returns
    (sorted cuts, normvec)."""
    p = int(np.sum(pvec))
    pst = block_starts(pvec)
    nv = block_normvec(R, pvec)
    cuts = {int(pst[j + 1]) for j in range(len(pvec) - 1) if nv[j] < tol}

    def split_largest():
        runs = _runs(cuts, p)
        a, b = max(runs, key=lambda r: (r[1] - r[0], -r[0]))
        if b - a >= 2:
            cuts.add(a + (b - a) // 2)

    if maxsize is not None:
        runs = _runs(cuts, p)
        if max(b - a for a, b in runs) > maxsize:
            split_largest()
    if numproc is not None:
        runs = _runs(cuts, p)
        if len(runs) > numproc:
            i = min(range(len(runs) - 1), key=lambda q: (runs[q + 1][1] - runs[q][0], q))
            cuts.discard(runs[i][1])
        elif len(runs) < numproc - 2:
            split_largest()
    return sorted(cuts), nv


def r_block(R: np.ndarray, pvec, tol: float, maxsize=None, numproc=None) -> np.ndarray:
    """Alg. 3: R_block = R inside each run, 0 between runs (block diagonal)."""
    p = R.shape[0]
    cuts, _ = r_block_cuts(R, pvec, tol, maxsize, numproc)
    run = np.searchsorted(np.asarray(cuts, dtype=np.int64), np.arange(p), side="right")
    return np.where(run[:, None] == run[None, :], R, 0.0)


def rhat(R: np.ndarray, kind: str, kappa_max: float = 100.0, block=None) -> np.ndarray:
    """R-hat of Sec. 5; ``block`` = (pvec, tol, maxsize, numproc) for "block"."""
    if kind == "exact":
        return R.copy()
    if kind == "rr":
        return r_ridge(R, kappa_max)[0]
    if kind == "me":
        return r_min_eig(R, kappa_max)[0]
    if kind == "diag":
        return r_diag(R)
    if kind == "block":
        pvec, tol, maxsize, numproc = block
        return r_block(R, pvec, tol, maxsize, numproc)
    raise ValueError(kind)


# ---------------------------------------- modified SOAR and channel-block R
def modified_soar_row(s: int, amp: float, length: float, maxval: int) -> np.ndarray:
    """First row of the banded circulant modified SOAR matrix (Sec. 6.1)."""
    maxval = int(maxval)
    if maxval < 1 or 2 * maxval + 1 > s:
        raise ValueError("modified SOAR needs 1 <= maxval and 2 maxval + 1 <= s")
    i = np.arange(-maxval, maxval + 1)
    d = 2.0 * np.abs(np.sin(i * (np.pi / maxval) / 2.0))
    row = np.zeros(s)
    row[i % s] = soar_function(d, amp, length)
    return row


def circulant(row: np.ndarray) -> np.ndarray:
    """C[j, k] = row[(k - j) mod s] (symmetric when row[i] = row[-i])."""
    s = row.size
    return row[(np.arange(s)[None, :] - np.arange(s)[:, None]) % s]


def modified_soar_shift(row: np.ndarray, psi: float) -> float:
    """|lambda_min| + psi when the circulant matrix of ``row`` has a negative
    eigenvalue, else 0.  The eigenvalues of a symmetric circulant matrix are
    the DFT of its first row."""
    lam_min = float(np.min(np.fft.fft(row).real))
    return abs(lam_min) + float(psi) if lam_min < 0.0 else 0.0


def modified_soar(s: int, amp: float, length: float, maxval: int, psi: float):
    """B or Q of the heat-equation experiments: (matrix, diagonal shift)."""
    row = modified_soar_row(s, amp, length, maxval)
    delta = modified_soar_shift(row, psi)
    return circulant(row) + delta * np.eye(s), delta


def modified_soar_apply(row: np.ndarray, delta: float, V: np.ndarray) -> np.ndarray:
    """(circulant(row) + delta I) V for V of shape [s] or [s, m], through the
    band only (for sizes where the dense matrix does not fit)."""
    s = row.size
    maxval = (np.count_nonzero(row) - 1) // 2
    out = delta * V
    for i in range(-maxval, maxval + 1):
        # (C V)_j = sum_i row[i] V_{j+i}
        out = out + row[i % s] * np.roll(V, -i, axis=0)
    return out


def pcorr_factors(draw_on: np.ndarray, draw_u: np.ndarray, pcorr_max: float, uncorrelated: float) -> np.ndarray:
    """pcorr of Sec. 6.1 from two uniform draws per pair of channel blocks:
    pcorr_max u where the first draw is at least ``uncorrelated``, else 0."""
    return np.where(draw_on >= uncorrelated, pcorr_max * draw_u, 0.0)


def block_r_matrix(pvec, density: float, pcorr: np.ndarray, u: np.ndarray, msoar, lmin: float) -> np.ndarray:
    """Channel-block R_i of Sec. 6.1.  ``u`` [p, p] uniform draws give the
    sparse random factors: entry (a, b) is u/density where u < density, else
    0.  Channel-block pairs (a, b), a < b, are numbered row by row.  A diagonal
    block of size m uses the modified SOAR with maxval min(msoar maxval,
    (m - 1) // 2) (no band when that is 0: amplitude on the diagonal)."""
    pvec = np.asarray(pvec, dtype=np.int64)
    pst = block_starts(pvec)
    p = int(pst[-1])
    S = np.where(u < density, u / density, 0.0)
    U = np.zeros((p, p))
    amp, length, maxval = msoar
    for k in range(len(pvec)):
        m = int(pvec[k])
        mv = min(int(maxval), (m - 1) // 2)
        C = circulant(modified_soar_row(m, amp, length, mv)) if mv >= 1 else amp * np.eye(m)
        sl = slice(pst[k], pst[k + 1])
        U[sl, sl] = S[sl, sl] * C
    q = 0
    for a in range(len(pvec)):
        for b in range(a + 1, len(pvec)):
            sa, sb = slice(pst[a], pst[a + 1]), slice(pst[b], pst[b + 1])
            U[sa, sb] = pcorr[q] * S[sa, sb]
            q += 1
    R = U + U.T
    lam_min = np.linalg.eigvalsh(R)[0]
    return R + (lmin - lam_min) * np.eye(p)


class SPDSolver:
    """x = M^{-1} v through a Cholesky factorisation (the exact-Cholesky
    reading of the paper's incomplete Cholesky on dense blocks)."""

    def __init__(self, M: np.ndarray):
        self.factor = sla.cho_factor(M, lower=True)

    def __call__(self, v: np.ndarray) -> np.ndarray:
        return sla.cho_solve(self.factor, v)
