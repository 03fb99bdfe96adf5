"""The saddle-point system of weak-constraint 4D-Var and its preconditioners.

Eq. saddlepointsystem / saddlepointA:

    A = [[D, 0, L], [0, R, H], [L^T, H^T, 0]],   unknowns (d_eta, d_nu, d_x),
    right-hand side (b, d, 0),

with D = blkdiag(B, Q_1..Q_N), R = blkdiag(R_0..R_N), H = blkdiag(H_0..H_N)
(Sec. 2.1).  Q_i = Q and R_i = R for every time (Sec. 6.1); H_i selects the
observed grid points (one unit entry per row, Sec. 6.1).

A vector is stored time-major: [eta (N+1) x s | nu (N+1) x p | x (N+1) x s].

Blockwise applies follow Sec. 6.2:
  A v      : c1 = D v1 + L v3,  c2 = R v2 + H v3,  c3 = L^T v1 + H^T v2
  P_D^{-1} v = (Dhat^{-1} v1, Rhat^{-1} v2, Shat^{-1} v3),
             Shat^{-1} = Lhat^{-1} D Lhat^{-T}  (paper's Schur approximation,
             Shat = Lhat^T D^{-1} Lhat, Sec. 2.2 / Sec. 3)
  P_I^{-1} v : c1 = Lhat^{-T} v3, c2 = Rhat^{-1} v2, c3 = Lhat^{-1}(v1 - D c1)
The exact negative Schur complement S = L^T D^{-1} L + H^T R^{-1} H (Sec. 2.2)
is available as Shat for small problems.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np
import scipy.linalg as sla

from . import covariance as cov
from . import model as mdl


@dataclass
class Problem:
    s: int
    N: int
    p: int
    model: object              # StencilModel / BandedModel
    obs_idx: np.ndarray        # [p] sorted observed grid indices
    B: np.ndarray
    Q: np.ndarray
    R: np.ndarray

    @property
    def n(self) -> int:
        return (2 * self.s + self.p) * (self.N + 1)

    def split(self, v: np.ndarray):
        s, p, T = self.s, self.p, self.N + 1
        v1 = v[:T * s].reshape(T, s)
        v2 = v[T * s:T * (s + p)].reshape(T, p)
        v3 = v[T * (s + p):].reshape(T, s)
        return v1, v2, v3

    @staticmethod
    def join(c1, c2, c3) -> np.ndarray:
        return np.concatenate([c1.ravel(), c2.ravel(), c3.ravel()])

    # ---- block operators on (N+1, .) arrays
    def D_apply(self, v1: np.ndarray) -> np.ndarray:
        out = np.empty_like(v1)
        out[0] = self.B @ v1[0]
        if self.N > 0:
            out[1:] = (self.Q @ v1[1:].T).T      # Q_i = Q for i = 1..N
        return out

    def R_apply(self, v2: np.ndarray) -> np.ndarray:
        return (self.R @ v2.T).T

    def H_apply(self, x: np.ndarray) -> np.ndarray:
        return x[:, self.obs_idx]

    def HT_apply(self, y: np.ndarray) -> np.ndarray:
        out = np.zeros((y.shape[0], self.s))
        out[:, self.obs_idx] = y
        return out

    # ---- Sec. 6.2: matrix-free A v
    def A_apply(self, v: np.ndarray) -> np.ndarray:
        v1, v2, v3 = self.split(v)
        c1 = self.D_apply(v1) + mdl.L_apply(self.model, v3)
        c2 = self.R_apply(v2) + self.H_apply(v3)
        c3 = mdl.LT_apply(self.model, v1) + self.HT_apply(v2)
        return self.join(c1, c2, c3)

    # ---- dense assembly (Eq. saddlepointA)
    def H_dense(self) -> np.ndarray:
        Hi = np.zeros((self.p, self.s))
        Hi[np.arange(self.p), self.obs_idx] = 1.0
        return np.kron(np.eye(self.N + 1), Hi)

    def D_dense(self) -> np.ndarray:
        return sla.block_diag(self.B, *([self.Q] * self.N))

    def R_dense(self) -> np.ndarray:
        return np.kron(np.eye(self.N + 1), self.R)

    def A_dense(self) -> np.ndarray:
        D, R, H = self.D_dense(), self.R_dense(), self.H_dense()
        L = mdl.L_dense(self.model)
        Z = np.zeros
        ns, npp = D.shape[0], R.shape[0]
        return np.block([[D, Z((ns, npp)), L],
                         [Z((npp, ns)), R, H],
                         [L.T, H.T, Z((ns, ns))]])

    def S_dense(self) -> np.ndarray:
        """Exact negative Schur complement S = L^T D^{-1} L + H^T R^{-1} H."""
        L = mdl.L_dense(self.model)
        D, R, H = self.D_dense(), self.R_dense(), self.H_dense()
        return L.T @ np.linalg.solve(D, L) + H.T @ np.linalg.solve(R, H)


@dataclass
class PrecondOptions:
    kind: str = "PD"          # "PD" (block diagonal) | "PI" (inexact constraint)
    k: int = 1                # Lhat = L_M(k); 1 -> L_0 = I, N+1 -> L
    rhat: str = "exact"       # "exact" | "rr" | "me" | "diag" | "block"
    rblock: tuple = ()        # "block": (pvec, tol, maxsize, numproc) of Alg. 3
    kappa_max: float = 100.0
    shat: str = "paper"       # "paper" (Lhat^T D^{-1} Lhat) | "exact" (S)
    dhat: str = "exact"       # "exact" | "rr"  (D + delta I, Sec. 6.1 delta = 0.01)
    dhat_delta: float = 0.01
    lhat_identity: bool = False   # L_I of Sec. 2.2 (M_t -> I inside Lhat)


class Counter:
    """Per-component product counts in the style of Tables 4 and 5: one count
    per time block touched (N+1 per full pass)."""

    def __init__(self):
        self.R = self.Rhat_inv = self.D = self.Dhat_inv = self.M = 0


class Preconditioner:
    def __init__(self, prob: Problem, opts: PrecondOptions, counter: Optional[Counter] = None):
        self.prob, self.o = prob, opts
        self.counter = counter
        N = prob.N
        if not (1 <= opts.k <= N + 1):
            raise ValueError("k must lie in [1, N+1]")
        self.lhat_model = mdl.IdentityModel(prob.s, N) if opts.lhat_identity else prob.model
        self._build_rhat()
        if opts.dhat == "exact":
            Bh, Qh = prob.B, prob.Q
        elif opts.dhat == "rr":
            Bh = prob.B + opts.dhat_delta * np.eye(prob.s)
            Qh = prob.Q + opts.dhat_delta * np.eye(prob.s)
        else:
            raise ValueError(opts.dhat)
        self.Bhat_solve = cov.SPDSolver(Bh) if opts.kind == "PD" else None
        self.Qhat_solve = cov.SPDSolver(Qh) if opts.kind == "PD" else None
        self.S_solve = cov.SPDSolver(prob.S_dense()) if opts.shat == "exact" else None

    def _build_rhat(self):
        o = self.o
        self.Rhat = cov.rhat(self.prob.R, o.rhat, o.kappa_max, o.rblock or None)
        self.Rhat_solve = cov.SPDSolver(self.Rhat)

    def Rhat_dense(self):
        return np.kron(np.eye(self.prob.N + 1), self.Rhat)

    # ---- pieces
    def Lhat_inv(self, v):
        return mdl.LM_inv(self.lhat_model, v, self.o.k)

    def Lhat_inv_T(self, v):
        return mdl.LM_inv_T(self.lhat_model, v, self.o.k)

    def Dhat_inv(self, v1):
        out = np.empty_like(v1)
        out[0] = self.Bhat_solve(v1[0])
        if self.prob.N > 0:
            out[1:] = self.Qhat_solve(v1[1:].T).T
        return out

    def Rhat_inv(self, v2):
        return self.Rhat_solve(v2.T).T

    def Shat_inv(self, v3):
        if self.S_solve is not None:
            return self.S_solve(v3.ravel()).reshape(v3.shape)
        return self.Lhat_inv(self.prob.D_apply(self.Lhat_inv_T(v3)))

    # ---- Sec. 6.2 applies
    def apply(self, v: np.ndarray) -> np.ndarray:
        p = self.prob
        v1, v2, v3 = p.split(v)
        if self.o.kind == "PD":
            return p.join(self.Dhat_inv(v1), self.Rhat_inv(v2), self.Shat_inv(v3))
        if self.o.kind == "PI":
            c1 = self.Lhat_inv_T(v3)
            c2 = self.Rhat_inv(v2)
            c3 = self.Lhat_inv(v1 - p.D_apply(c1))
            return p.join(c1, c2, c3)
        raise ValueError(self.o.kind)

    # ---- dense forms (Eq. prec) for the pins
    def Lhat_dense(self):
        return mdl.LM_dense(self.lhat_model, self.o.k)

    def Dhat_dense(self):
        p = self.prob
        if self.o.dhat == "exact":
            return p.D_dense()
        return p.D_dense() + self.o.dhat_delta * np.eye(p.s * (p.N + 1))

    def Shat_dense(self):
        p = self.prob
        if self.o.shat == "exact":
            return p.S_dense()
        Lh = self.Lhat_dense()
        return Lh.T @ np.linalg.solve(p.D_dense(), Lh)

    def dense(self) -> np.ndarray:
        p = self.prob
        Rh = self.Rhat_dense()
        ns, npp = p.s * (p.N + 1), Rh.shape[0]
        Z = np.zeros
        if self.o.kind == "PD":
            return sla.block_diag(self.Dhat_dense(), Rh, self.Shat_dense())
        Lh = self.Lhat_dense()
        return np.block([[p.D_dense(), Z((ns, npp)), Lh],
                         [Z((npp, ns)), Rh, Z((npp, ns))],
                         [Lh.T, Z((ns, npp)), Z((ns, ns))]])


# ------------------------------------------- per-time observations (H_i, R_i)
class PerTimeProblem(Problem):
    """The general blocks of Sec. 2.1: time i observes the p_i grid points
    obs_list[i] (H_i selects them) with its own error covariance R_list[i];
    R = blkdiag(R_0..R_N), H = blkdiag(H_0..H_N).  nu is stored as the
    concatenation of the N+1 blocks of sizes p_i, so ``split`` returns it as a
    list.  ``p`` is the total number of observations over the window."""

    def __init__(self, s, N, model, obs_list, B, Q, R_list):
        if len(obs_list) != N + 1 or len(R_list) != N + 1:
            raise ValueError("need N+1 observation sets and R_i blocks")
        self.s, self.N, self.model, self.B, self.Q = s, N, model, B, Q
        self.obs_list = [np.asarray(o) for o in obs_list]
        self.R_list = [np.asarray(r, dtype=np.float64) for r in R_list]
        self.p_list = [len(o) for o in self.obs_list]
        for o, r in zip(self.obs_list, self.R_list):
            if r.shape != (len(o), len(o)):
                raise ValueError("R_i must be p_i x p_i")
        self.p = int(sum(self.p_list))
        self.obs_idx = None
        self.R = None

    @property
    def n(self) -> int:
        return 2 * self.s * (self.N + 1) + self.p

    def split(self, v: np.ndarray):
        s, T = self.s, self.N + 1
        v1 = v[:T * s].reshape(T, s)
        off = T * s
        v2 = []
        for pi in self.p_list:
            v2.append(v[off:off + pi])
            off += pi
        v3 = v[off:].reshape(T, s)
        return v1, v2, v3

    @staticmethod
    def join(c1, c2, c3) -> np.ndarray:
        return np.concatenate([c1.ravel()] + [np.ravel(x) for x in c2] + [c3.ravel()])

    def R_apply(self, v2):
        return [Ri @ vi for Ri, vi in zip(self.R_list, v2)]

    def A_apply(self, v: np.ndarray) -> np.ndarray:
        v1, v2, v3 = self.split(v)
        c1 = self.D_apply(v1) + mdl.L_apply(self.model, v3)
        c2 = [r + h for r, h in zip(self.R_apply(v2), self.H_apply(v3))]
        c3 = mdl.LT_apply(self.model, v1) + self.HT_apply(v2)
        return self.join(c1, c2, c3)

    def H_apply(self, x: np.ndarray):
        return [x[i, o] for i, o in enumerate(self.obs_list)]

    def HT_apply(self, y) -> np.ndarray:
        out = np.zeros((self.N + 1, self.s))
        for i, o in enumerate(self.obs_list):
            out[i, o] = y[i]
        return out

    def H_dense(self) -> np.ndarray:
        blocks = []
        for o in self.obs_list:
            Hi = np.zeros((len(o), self.s))
            Hi[np.arange(len(o)), o] = 1.0
            blocks.append(Hi)
        return sla.block_diag(*blocks)

    def R_dense(self) -> np.ndarray:
        return sla.block_diag(*self.R_list)


class BandCovProblem(Problem):
    """The heat-equation window at sizes where dense B and Q do not fit
    (Sec. 7.2: s up to 50,000): B and Q are the banded circulant modified SOAR
    of Sec. 6.1, stored as their first rows plus the diagonal shifts, and
    applied through the band (cov.modified_soar_apply, pinned against the dense
    circulant product).  Everything else is the shared-set Problem; the dense
    assemblies that need B or Q are not available."""

    def __init__(self, s, N, p, model, obs_idx, rowB, deltaB, rowQ, deltaQ, R):
        super().__init__(s, N, p, model, obs_idx, None, None, R)
        self.rowB, self.deltaB, self.rowQ, self.deltaQ = rowB, deltaB, rowQ, deltaQ

    def D_apply(self, v1: np.ndarray) -> np.ndarray:
        out = np.empty_like(v1)
        out[0] = cov.modified_soar_apply(self.rowB, self.deltaB, v1[0])
        if self.N > 0:
            out[1:] = cov.modified_soar_apply(self.rowQ, self.deltaQ, v1[1:].T).T
        return out


class PerTimePreconditioner(Preconditioner):
    """P_D / P_I (Eq. prec) with R-hat_i built from each R_i (Sec. 5 applied
    blockwise, as the paper's Remark in Sec. 5 states)."""

    def _build_rhat(self):
        o = self.o
        self.Rhat_list = [cov.rhat(Ri, o.rhat, o.kappa_max, o.rblock or None) for Ri in self.prob.R_list]
        self.Rhat_solves = [cov.SPDSolver(Rh) for Rh in self.Rhat_list]

    def Rhat_dense(self):
        return sla.block_diag(*self.Rhat_list)

    def Rhat_inv(self, v2):
        return [solve(vi) for solve, vi in zip(self.Rhat_solves, v2)]


# ------------------------------------------------------------ direct solves
def dense_solve(prob: Problem, rhs: np.ndarray) -> np.ndarray:
    """LU with partial pivoting of the assembled A (feasible for n <~ 8000)."""
    A = prob.A_dense()
    lu, piv = sla.lu_factor(A)
    return sla.lu_solve((lu, piv), rhs)


def primal_solve(prob: Problem, b: np.ndarray, d: np.ndarray):
    """Primal check: the minimiser of the linearised cost
        J(dx) = ||L dx - b||^2_{D^{-1}} + ||H dx - d||^2_{R^{-1}}
    solves S dx = L^T D^{-1} b + H^T R^{-1} d; then eta = D^{-1}(b - L dx) and
    nu = R^{-1}(d - H dx) (block rows of Eq. saddlepointsystem)."""
    L = mdl.L_dense(prob.model)
    D, R, H = prob.D_dense(), prob.R_dense(), prob.H_dense()
    Dinv_b = np.linalg.solve(D, b)
    Rinv_d = np.linalg.solve(R, d)
    S = prob.S_dense()
    dx = np.linalg.solve(S, L.T @ Dinv_b + H.T @ Rinv_d)
    eta = np.linalg.solve(D, b - L @ dx)
    nu = np.linalg.solve(R, d - H @ dx)
    return np.concatenate([eta, nu, dx])


def linearised_cost(prob: Problem, b: np.ndarray, d: np.ndarray, dx: np.ndarray) -> float:
    """J_lin(dx) of the inner loop (Eq. CostFn linearised; no 1/2 factors)."""
    L = mdl.L_dense(prob.model)
    D, R, H = prob.D_dense(), prob.R_dense(), prob.H_dense()
    e1 = L @ dx - b
    e2 = H @ dx - d
    return float(e1 @ np.linalg.solve(D, e1) + e2 @ np.linalg.solve(R, e2))
