"""Model matrices M_i, the block model matrix L and its approximations.

Indexing: time levels t = 0..N (0-based).  M_t (t = 1..N) maps time t-1 to
time t, matching Eq. def:L where block row t carries -M_t in block column t-1.

* L (Eq. def:L):             (L z)_t = z_t - M_t z_{t-1}            (t >= 1)
* L_M(k) (Definition 1):     the sub-diagonal block -M_j is dropped when j is
  divisible by k.  With t = j (0-based row t = j), the coupling into time t is
  kept iff t mod k != 0, so time levels split into the independent chunks
  {0..k-1}, {k..2k-1}, ...  L_M(1) = I (= L_0, Sec. 2.2), L_M(N+1) = L.
* Lemma 1: inside a chunk, block (t, u) of L_M^{-1} is M_t M_{t-1} ... M_{u+1}
  (M_{u+1} acts first).  Applying it is the forward recursion
  z_t = v_t + [t mod k != 0] M_t z_{t-1}; the transpose runs backward,
  z_t = v_t + [(t+1) mod k != 0] M_{t+1}^T z_{t+1}.
* L_I (Sec. 2.2): every M_t replaced by the identity.

Advection-diffusion (linear workloads): one explicit step of periodic upwind
advection (Courant c) plus central diffusion (number d):
  (M x)_j = (c+d) x_{j-1} + (1-c-2d) x_j + d x_{j+1}.
Heat equation (Sec. 7.2): Dirichlet boundaries, stored banded (heat_model).
Lorenz-96 (Sec. 7.1): dx_j/dt = (x_{j+1} - x_{j-2}) x_{j-1} - x_j + F, periodic,
integrated with classical RK4; M_i is the exact chain-rule Jacobian of the
``steps_per_obs`` RK4 steps between two observation times, stored banded.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


# ----------------------------------------------------------------- operators
class StencilModel:
    """M_t = the same periodic 3-point stencil for every t (linear model)."""

    def __init__(self, s: int, N: int, coeffs):
        self.s, self.N = s, N
        self.cl, self.cm, self.cr = (float(c) for c in coeffs)

    def apply(self, t: int, x: np.ndarray) -> np.ndarray:
        return self.cl * np.roll(x, 1) + self.cm * x + self.cr * np.roll(x, -1)

    def apply_T(self, t: int, y: np.ndarray) -> np.ndarray:
        # (M^T y)_j = cl y_{j+1} + cm y_j + cr y_{j-1}
        return self.cl * np.roll(y, -1) + self.cm * y + self.cr * np.roll(y, 1)

    def dense(self, t: int) -> np.ndarray:
        s = self.s
        M = np.zeros((s, s))
        j = np.arange(s)
        M[j, (j - 1) % s] += self.cl
        M[j, j] += self.cm
        M[j, (j + 1) % s] += self.cr
        return M


class BandedModel:
    """M_t stored as bands: bands[t-1, j, o+lo] = M_t[j, (j+o) mod s], o in [-lo, hi]."""

    def __init__(self, bands: np.ndarray, lo: int, hi: int):
        self.bands = np.asarray(bands, dtype=np.float64)
        self.N, self.s, w = self.bands.shape
        assert w == lo + hi + 1
        if w > self.s:
            raise ValueError("band wider than the state: offsets would alias modulo s")
        self.lo, self.hi = lo, hi
        self._csr = {}

    def csr(self, t: int) -> sp.csr_matrix:
        if t not in self._csr:
            s = self.s
            rows, cols, vals = [], [], []
            j = np.arange(s)
            for o in range(-self.lo, self.hi + 1):
                rows.append(j)
                cols.append((j + o) % s)
                vals.append(self.bands[t - 1, :, o + self.lo])
            M = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                              shape=(s, s)).tocsr()
            self._csr[t] = M
        return self._csr[t]

    def apply(self, t: int, x: np.ndarray) -> np.ndarray:
        return self.csr(t) @ x

    def apply_T(self, t: int, y: np.ndarray) -> np.ndarray:
        return self.csr(t).T @ y

    def dense(self, t: int) -> np.ndarray:
        return self.csr(t).toarray()


class IdentityModel:
    """M_t = I for every t: the L_I approximation of Sec. 2.2."""

    def __init__(self, s: int, N: int):
        self.s, self.N = s, N

    def apply(self, t, x):
        return x.copy()

    def apply_T(self, t, y):
        return y.copy()

    def dense(self, t):
        return np.eye(self.s)


def heat_model(s: int, N: int, r: float) -> BandedModel:
    """Sec. 7.2: the heat equation on the unit line, forward Euler in time and
    centred differences in space, homogeneous Dirichlet boundaries: the two
    boundary rows and columns of M are zero and interior row j carries
    (r, 1 - 2r, r) on columns j-1, j, j+1 (the couplings into the boundary
    columns 0 and s-1 are zero), r = alpha dt / dx^2."""
    if s < 3:
        raise ValueError("the heat model needs s >= 3")
    bands = np.zeros((N, s, 3))
    j = np.arange(1, s - 1)
    bands[:, j, 0] = np.where(j - 1 >= 1, r, 0.0)
    bands[:, j, 1] = 1.0 - 2.0 * r
    bands[:, j, 2] = np.where(j + 1 <= s - 2, r, 0.0)
    return BandedModel(bands, 1, 1)


def advdiff_coeffs(courant: float, diffusion: float):
    c, d = courant, diffusion
    return (c + d, 1.0 - c - 2.0 * d, d)


# --------------------------------------------------------- L and L_M(k)
def keeps_coupling(t: int, k: int) -> bool:
    """Definition 1: the block -M_t (into time t) survives iff t mod k != 0."""
    return t % k != 0


def L_apply(model, z: np.ndarray) -> np.ndarray:
    """Eq. def:L acting on z of shape (N+1, s)."""
    out = z.copy()
    for t in range(1, model.N + 1):
        out[t] -= model.apply(t, z[t - 1])
    return out


def LT_apply(model, y: np.ndarray) -> np.ndarray:
    out = y.copy()
    for t in range(0, model.N):
        out[t] -= model.apply_T(t + 1, y[t + 1])
    return out


def LM_apply(model, z: np.ndarray, k: int) -> np.ndarray:
    """L_M(k) z (Definition 1)."""
    out = z.copy()
    for t in range(1, model.N + 1):
        if keeps_coupling(t, k):
            out[t] -= model.apply(t, z[t - 1])
    return out


def LM_inv(model, v: np.ndarray, k: int) -> np.ndarray:
    """L_M(k)^{-1} v by the forward recursion of Lemma 1."""
    z = v.copy()
    for t in range(1, model.N + 1):
        if keeps_coupling(t, k):
            z[t] = v[t] + model.apply(t, z[t - 1])
    return z


def LM_inv_T(model, v: np.ndarray, k: int) -> np.ndarray:
    """L_M(k)^{-T} v by the backward recursion."""
    z = v.copy()
    for t in range(model.N - 1, -1, -1):
        if keeps_coupling(t + 1, k):
            z[t] = v[t] + model.apply_T(t + 1, z[t + 1])
    return z


def L_dense(model) -> np.ndarray:
    return LM_dense(model, model.N + 1)


def LM_dense(model, k: int) -> np.ndarray:
    s, N = model.s, model.N
    L = np.eye((N + 1) * s)
    for t in range(1, N + 1):
        if keeps_coupling(t, k):
            L[t * s:(t + 1) * s, (t - 1) * s:t * s] = -model.dense(t)
    return L


def lemma1_block(model, k: int, i: int, j: int) -> np.ndarray:
    """Lemma 1 (1-based block indices i, j = 1..N+1): block (i, j) of L_M^{-1}
    is I for i = j, the product M_{i-1} M_{i-2} ... M_j for
    1 <= i-j <= (i-1) mod k, and zero otherwise."""
    s = model.s
    if i == j:
        return np.eye(s)
    if 1 <= i - j <= (i - 1) % k:
        P = np.eye(s)
        for m in range(1, i - j + 1):     # left factor first: M_{i-1}, then M_{i-2} ...
            P = P @ model.dense(i - m)
        return P
    return np.zeros((s, s))


# ---------------------------------------------------------------- Lorenz-96
def l96_rhs(x: np.ndarray, F: float) -> np.ndarray:
    return (np.roll(x, -1) - np.roll(x, 2)) * np.roll(x, 1) - x + F


def rk4_step(x: np.ndarray, dt: float, F: float) -> np.ndarray:
    k1 = l96_rhs(x, F)
    k2 = l96_rhs(x + 0.5 * dt * k1, F)
    k3 = l96_rhs(x + 0.5 * dt * k2, F)
    k4 = l96_rhs(x + dt * k3, F)
    return x + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


def l96_forecast(x: np.ndarray, dt: float, F: float, steps: int) -> np.ndarray:
    for _ in range(steps):
        x = rk4_step(x, dt, F)
    return x


def l96_jacobian(x: np.ndarray) -> sp.csr_matrix:
    """d f / d x for the Lorenz-96 right-hand side (4 non-zeros per row)."""
    s = x.size
    j = np.arange(s)
    rows = np.concatenate([j, j, j, j])
    cols = np.concatenate([(j + 1) % s, (j - 2) % s, (j - 1) % s, j])
    vals = np.concatenate([np.roll(x, 1),                      # d/dx_{j+1} = x_{j-1}
                           -np.roll(x, 1),                     # d/dx_{j-2} = -x_{j-1}
                           np.roll(x, -1) - np.roll(x, 2),     # d/dx_{j-1} = x_{j+1} - x_{j-2}
                           -np.ones(s)])                       # d/dx_j = -1
    return sp.coo_matrix((vals, (rows, cols)), shape=(s, s)).tocsr()


def rk4_step_tlm(x: np.ndarray, dt: float, F: float) -> sp.csr_matrix:
    """Exact Jacobian of one RK4 step about x (chain rule through the stages)."""
    s = x.size
    I = sp.identity(s, format="csr")
    k1 = l96_rhs(x, F)
    x2 = x + 0.5 * dt * k1
    k2 = l96_rhs(x2, F)
    x3 = x + 0.5 * dt * k2
    k3 = l96_rhs(x3, F)
    x4 = x + dt * k3
    K1 = l96_jacobian(x)
    K2 = l96_jacobian(x2) @ (I + 0.5 * dt * K1)
    K3 = l96_jacobian(x3) @ (I + 0.5 * dt * K2)
    K4 = l96_jacobian(x4) @ (I + dt * K3)
    return (I + (dt / 6.0) * (K1 + 2.0 * K2 + 2.0 * K3 + K4)).tocsr()


def l96_tlm(x: np.ndarray, dt: float, F: float, steps: int) -> sp.csr_matrix:
    """Jacobian of ``steps`` RK4 steps starting at x (later steps act last)."""
    M = sp.identity(x.size, format="csr")
    for _ in range(steps):
        M = rk4_step_tlm(x, dt, F) @ M
        x = rk4_step(x, dt, F)
    return M.tocsr()


def band_width(steps: int):
    """Offsets of a steps-long RK4 Jacobian: each stage couples j-2..j+1, four
    stages per step, so one step spans -8..+4 and ``steps`` steps -8s..+4s."""
    return 8 * steps, 4 * steps


def to_bands(M: sp.spmatrix, lo: int, hi: int) -> np.ndarray:
    """Extract bands[j, o+lo] = M[j, (j+o) mod s]; entries outside the band must be 0."""
    D = M.toarray()
    s = D.shape[0]
    if lo + hi + 1 > s:
        raise ValueError("band wider than the state: offsets would alias modulo s")
    out = np.zeros((s, lo + hi + 1))
    j = np.arange(s)
    mask = np.zeros_like(D, dtype=bool)
    for o in range(-lo, hi + 1):
        out[:, o + lo] = D[j, (j + o) % s]
        mask[j, (j + o) % s] = True
    if np.any(D[~mask] != 0.0):
        raise ValueError("matrix has entries outside the declared band")
    return out
