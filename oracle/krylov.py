"""Krylov solvers for the saddle-point system (Sec. 2.1, Sec. 7).

* MINRES with a symmetric positive definite preconditioner (the block-diagonal
  P_D), in the preconditioned Lanczos form of Elman-Silvester-Wathen (2014),
  Ch. 4, which the paper cites for the convergence theory (Sec. 3).  The
  recurrence carries eta with |eta_j| = ||r_j||_{P^{-1}}.
* GMRES with right preconditioning and no restarts (Sec. 7 uses GMRES without
  restarts for the inexact-constraint P_I), Arnoldi by modified Gram-Schmidt,
  Givens rotations on the Hessenberg matrix; |g_{j+1}| = ||r_j||_2.
* FGMRES (flexible, right-preconditioned): the same with the preconditioned
  basis vectors Z stored, so the preconditioner may change per iteration.

Stopping (Sec. 6.2 / Sec. 7): relative residual 1e-6 in the 2-norm, at most
1000 iterations.  MINRES triggers on its recurrence estimate and then accepts
only when the true FP64 relative residual ||rhs - A x||_2 / ||rhs||_2 <= tol;
otherwise it continues (reading of the "residual-based criterion in the two
norm").
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np


@dataclass
class KrylovResult:
    x: np.ndarray
    iters: int
    converged: bool
    relres_true: float
    history: List[float] = field(default_factory=list)   # per-iteration residual estimate (relative)


def _true_relres(A, b, x):
    nb = np.linalg.norm(b)
    return np.linalg.norm(b - A(x)) / (nb if nb > 0 else 1.0)


def minres(A: Callable, Pinv: Callable, b: np.ndarray, x0: Optional[np.ndarray] = None,
           tol: float = 1e-6, maxit: int = 1000, check_true: bool = True) -> KrylovResult:
    n = b.size
    x = np.zeros(n) if x0 is None else x0.copy()
    v = b - A(x) if x0 is not None else b.copy()
    v_old = np.zeros(n)
    z = Pinv(v)
    gamma = np.sqrt(np.dot(z, v))
    gamma_old = 1.0
    eta = gamma
    eta0 = gamma if gamma > 0 else 1.0
    c_old = c = 1.0
    s_old = s = 0.0
    w_old = np.zeros(n)
    w = np.zeros(n)
    hist = []
    nb = np.linalg.norm(b)
    if nb == 0:
        return KrylovResult(x, 0, True, 0.0, hist)
    for j in range(1, maxit + 1):
        z = z / gamma
        Az = A(z)
        delta = np.dot(Az, z)
        v_new = Az - (delta / gamma) * v - (gamma / gamma_old) * v_old
        z_new = Pinv(v_new)
        gamma_new = np.sqrt(max(np.dot(z_new, v_new), 0.0))
        a0 = c * delta - c_old * s * gamma
        a1 = np.hypot(a0, gamma_new)
        a2 = s * delta + c_old * c * gamma
        a3 = s_old * gamma
        c_new = a0 / a1
        s_new = gamma_new / a1
        w_new = (z - a3 * w_old - a2 * w) / a1
        x = x + (c_new * eta) * w_new
        eta = -s_new * eta
        hist.append(abs(eta) / eta0)
        v_old, v = v, v_new
        z = z_new
        gamma_old, gamma = gamma, gamma_new
        c_old, c = c, c_new
        s_old, s = s, s_new
        w_old, w = w, w_new
        if abs(eta) / eta0 <= tol or gamma == 0.0:
            rr = _true_relres(A, b, x)
            if not check_true or rr <= tol or gamma == 0.0:
                return KrylovResult(x, j, rr <= tol, rr, hist)
    return KrylovResult(x, maxit, False, _true_relres(A, b, x), hist)


def _givens(a: float, b: float):
    if b == 0.0:
        return 1.0, 0.0
    r = np.hypot(a, b)
    return a / r, b / r


def gmres(A: Callable, Pinv: Callable, b: np.ndarray, x0: Optional[np.ndarray] = None,
          tol: float = 1e-6, maxit: int = 1000, flexible: bool = False) -> KrylovResult:
    """Right-preconditioned (F)GMRES without restarts.  ``Pinv`` may be a
    callable ``Pinv(v, j)`` when ``flexible`` (the preconditioner may vary)."""
    n = b.size
    x0 = np.zeros(n) if x0 is None else x0.copy()
    r0 = b - A(x0)
    beta = np.linalg.norm(r0)
    nb = np.linalg.norm(b)
    nb = nb if nb > 0 else 1.0
    if beta == 0.0:
        return KrylovResult(x0, 0, True, 0.0, [])
    V = [r0 / beta]
    Z = []
    Hm = np.zeros((maxit + 1, maxit))
    cs, sn = np.zeros(maxit), np.zeros(maxit)
    g = np.zeros(maxit + 1)
    g[0] = beta
    hist = []
    j_done = 0
    for j in range(maxit):
        zj = Pinv(V[j], j) if flexible else Pinv(V[j])
        Z.append(zj)
        w = A(zj)
        for i in range(j + 1):                      # modified Gram-Schmidt
            Hm[i, j] = np.dot(w, V[i])
            w = w - Hm[i, j] * V[i]
        Hm[j + 1, j] = np.linalg.norm(w)
        for i in range(j):                          # previous rotations
            t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
            Hm[i + 1, j] = -sn[i] * Hm[i, j] + cs[i] * Hm[i + 1, j]
            Hm[i, j] = t
        cs[j], sn[j] = _givens(Hm[j, j], Hm[j + 1, j])
        Hm[j, j] = cs[j] * Hm[j, j] + sn[j] * Hm[j + 1, j]
        Hm[j + 1, j] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        hist.append(abs(g[j + 1]) / nb)
        j_done = j + 1
        h_next = np.linalg.norm(w)
        if abs(g[j + 1]) / nb <= tol or h_next == 0.0:
            break
        V.append(w / h_next)
    k = j_done
    y = np.linalg.solve(np.triu(Hm[:k, :k]), g[:k])
    x = x0 + sum(y[i] * Z[i] for i in range(k))
    rr = _true_relres(A, b, x)
    return KrylovResult(x, k, rr <= tol, rr, hist)
