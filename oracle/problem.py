"""Synthetic problems, right-hand sides and the incremental outer loop.

Readings (the paper does not define them):
* C1 right-hand side.  For outer loop l about the trajectory x^(l), the
  linearised cost of Eq. CostFn gives
      b_0 = x_b - x_0^(l),   b_i = M_i(x_{i-1}^(l)) - x_i^(l),
      d_i = y_i - H_i(x_i^(l)),
  and the inner system is Eq. saddlepointsystem with right-hand side (b, d, 0).
  The first outer loop starts from the background forecast x^(0), so for a
  linear model b = 0 there.
* C17 truth and noise.  Linear workloads: truth x_0^t is a unit Gaussian bump,
  propagated by the perfect model; x_b = x_0^t + chol(B) z_b;
  y_i = H x_i^t + chol(R) z_i.  Lorenz-96: x_0^t = F + 0.01 z spun up by
  ``spinup_steps`` RK4 steps; truth model error chol(Q) z_i is added after each
  forecast between observation times.
* Sec. 2.1: x^(l+1) = x^(l) + dx^(l) over the whole window (weak constraint).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np
import scipy.linalg as sla

from . import covariance as cov
from . import model as mdl
from .saddle import BandCovProblem, PerTimeProblem, Problem, Preconditioner, PrecondOptions
from . import krylov
from paper_2105_06975_gb300 import workload


def covariances(w, obs_idx, extra=None):
    """B, Q and R_i of a workload: chordal SOAR (all but the heat workload) or
    the modified SOAR B, Q and the channel-block R_i of Sec. 6.1 (their draws
    in ``extra``)."""
    if w.cov == "msoar":
        B = cov.modified_soar(w.s, *w.msoar_b, extra["psi"][0])[0]
        Q = cov.modified_soar(w.s, *w.msoar_q, extra["psi"][1])[0]
    else:
        B = cov.soar_state(w.s, *w.soar_b)
        Q = cov.soar_state(w.s, *w.soar_q)
    return B, Q, observation_covariance(w, obs_idx, extra)


def observation_covariance(w, obs_idx, extra=None):
    """R_i of a workload: the channel-block R of Sec. 6.1 or the chordal SOAR
    over the observed points."""
    if w.r_kind == "block":
        pvec = workload.block_sizes(w.p, w.r_blocks)
        pcorr = cov.pcorr_factors(extra["pcorr_on"], extra["pcorr_u"], w.r_pcorr_max, w.r_uncorrelated)
        return cov.block_r_matrix(pvec, w.r_density, pcorr, extra["r_u"], w.r_msoar, w.r_lmin)
    return cov.soar_obs(w.s, obs_idx, *w.soar_r)


def linear_model(w):
    if w.model == "heat":
        return mdl.heat_model(w.s, w.N, w.heat_r)
    return mdl.StencilModel(w.s, w.N, mdl.advdiff_coeffs(w.courant, w.diffusion))


def linear_problem(w, dr) -> Problem:
    B, Q, R = covariances(w, dr.obs_idx, dr.extra)
    return Problem(w.s, w.N, w.p, linear_model(w), np.asarray(dr.obs_idx), B, Q, R)


def heat_band_problem(w, dr, R=None) -> BandCovProblem:
    """The heat workload with B and Q kept as their modified SOAR rows and
    shifts (Sec. 6.1, 7.2); R is the workload's R (channel-block or SOAR over
    the observed points) unless given."""
    rowB = cov.modified_soar_row(w.s, *w.msoar_b)
    rowQ = cov.modified_soar_row(w.s, *w.msoar_q)
    dB = cov.modified_soar_shift(rowB, dr.extra["psi"][0])
    dQ = cov.modified_soar_shift(rowQ, dr.extra["psi"][1])
    if R is None:
        R = observation_covariance(w, dr.obs_idx, dr.extra)
    return BandCovProblem(w.s, w.N, w.p, linear_model(w), np.asarray(dr.obs_idx), rowB, dB, rowQ, dQ, R)


def per_time_problem(w, dr) -> PerTimeProblem:
    """Distinct H_i, R_i per time: R_i is the workload's R over time i's
    observed points (chordal SOAR at obs_list[i]/s)."""
    B, Q, _ = covariances(w, dr.obs_idx, dr.extra)
    obs_list = dr.extra["obs_list"]
    R_list = [cov.soar_obs(w.s, o, *w.soar_r) for o in obs_list]
    return PerTimeProblem(w.s, w.N, linear_model(w), obs_list, B, Q, R_list)


def per_time_case(w, dr):
    """Problem, truth / observations and the first-loop right-hand side (C1,
    C17) with y_i = H_i x_i^t + chol(R_i) z_i."""
    prob = per_time_problem(w, dr)
    x0t = workload.bump(w, dr.bump_center)
    truth = np.zeros((w.N + 1, w.s))
    truth[0] = x0t
    for t in range(1, w.N + 1):
        truth[t] = prob.model.apply(t, truth[t - 1])
    xb = x0t + chol_lower(prob.B) @ dr.z_b
    y = [truth[i, o] + chol_lower(Ri) @ dr.z_r[i] for i, (o, Ri) in enumerate(zip(prob.obs_list, prob.R_list))]
    traj = background_trajectory_linear(prob, xb)
    b = np.zeros((w.N + 1, w.s))
    b[0] = xb - traj[0]
    d = [y[i] - traj[i, o] for i, o in enumerate(prob.obs_list)]
    rhs = PerTimeProblem.join(b, d, np.zeros((w.N + 1, w.s)))
    return prob, Observations(xb, y, truth), rhs


def chol_lower(M):
    return np.linalg.cholesky(M)


@dataclass
class Observations:
    xb: np.ndarray          # [s]
    y: np.ndarray           # [N+1, p]
    truth: np.ndarray       # [N+1, s]


def linear_observations(w, dr, prob: Problem) -> Observations:
    x0t = workload.bump(w, dr.bump_center)
    truth = np.zeros((w.N + 1, w.s))
    truth[0] = x0t
    for t in range(1, w.N + 1):
        truth[t] = prob.model.apply(t, truth[t - 1])
    xb = x0t + chol_lower(prob.B) @ dr.z_b
    LR = chol_lower(prob.R)
    y = truth[:, prob.obs_idx] + (LR @ dr.z_r.T).T
    return Observations(xb, y, truth)


def background_trajectory_linear(prob: Problem, xb):
    x = np.zeros((prob.N + 1, prob.s))
    x[0] = xb
    for t in range(1, prob.N + 1):
        x[t] = prob.model.apply(t, x[t - 1])
    return x


def rhs_linear(prob: Problem, obs: Observations, traj: np.ndarray) -> np.ndarray:
    """(b, d, 0) about the trajectory ``traj`` (C1) for a linear model."""
    b = np.zeros((prob.N + 1, prob.s))
    b[0] = obs.xb - traj[0]
    for t in range(1, prob.N + 1):
        b[t] = prob.model.apply(t, traj[t - 1]) - traj[t]
    d = obs.y - traj[:, prob.obs_idx]
    return Problem.join(b, d, np.zeros((prob.N + 1, prob.s)))


def linear_case(w, dr):
    prob = linear_problem(w, dr)
    obs = linear_observations(w, dr, prob)
    traj = background_trajectory_linear(prob, obs.xb)
    return prob, obs, rhs_linear(prob, obs, traj)


# ------------------------------------------------------------------ Lorenz-96
def l96_truth(w, dr, B, Q, R, obs_idx) -> Observations:
    x = w.forcing + 0.01 * dr.x0_pert
    x = mdl.l96_forecast(x, w.dt, w.forcing, w.spinup_steps)
    truth = np.zeros((w.N + 1, w.s))
    truth[0] = x
    LQ = chol_lower(Q)
    for t in range(1, w.N + 1):
        truth[t] = mdl.l96_forecast(truth[t - 1], w.dt, w.forcing, w.steps_per_obs) + LQ @ dr.z_q[t - 1]
    xb = truth[0] + chol_lower(B) @ dr.z_b
    y = truth[:, obs_idx] + (chol_lower(R) @ dr.z_r.T).T
    return Observations(xb, y, truth)


def l96_linearise(w, traj: np.ndarray):
    """Banded tangent-linear models M_1..M_N about traj[0..N-1] (C16)."""
    lo, hi = mdl.band_width(w.steps_per_obs)
    bands = np.zeros((w.N, w.s, lo + hi + 1))
    for t in range(1, w.N + 1):
        M = mdl.l96_tlm(traj[t - 1], w.dt, w.forcing, w.steps_per_obs)
        bands[t - 1] = mdl.to_bands(M, lo, hi)
    return bands, lo, hi


def l96_rhs(w, prob: Problem, obs: Observations, traj: np.ndarray) -> np.ndarray:
    b = np.zeros((w.N + 1, w.s))
    b[0] = obs.xb - traj[0]
    for t in range(1, w.N + 1):
        b[t] = mdl.l96_forecast(traj[t - 1], w.dt, w.forcing, w.steps_per_obs) - traj[t]
    d = obs.y - traj[:, prob.obs_idx]
    return Problem.join(b, d, np.zeros((w.N + 1, w.s)))


def l96_background(w, xb):
    traj = np.zeros((w.N + 1, w.s))
    traj[0] = xb
    for t in range(1, w.N + 1):
        traj[t] = mdl.l96_forecast(traj[t - 1], w.dt, w.forcing, w.steps_per_obs)
    return traj


def solve_inner(prob: Problem, rhs: np.ndarray, popts: PrecondOptions, krylov_kind: str,
                tol=1e-6, maxit=1000):
    P = Preconditioner(prob, popts)
    if krylov_kind == "minres":
        return krylov.minres(prob.A_apply, P.apply, rhs, tol=tol, maxit=maxit)
    if krylov_kind == "gmres":
        return krylov.gmres(prob.A_apply, P.apply, rhs, tol=tol, maxit=maxit)
    raise ValueError(krylov_kind)


def gauss_newton_l96(w, dr, popts: PrecondOptions, krylov_kind="gmres", tol=1e-6, maxit=1000,
                     loops: Optional[int] = None, obs: Optional[Observations] = None):
    """Incremental weak-constraint 4D-Var (Sec. 2.1) for Lorenz-96: each outer
    loop linearises about x^(l), solves the saddle-point inner problem and
    updates the whole trajectory.  Returns (trajectories, inner results)."""
    B, Q, R = covariances(w, dr.obs_idx)
    if obs is None:
        obs = l96_truth(w, dr, B, Q, R, dr.obs_idx)
    traj = l96_background(w, obs.xb)
    trajs, results = [traj.copy()], []
    for _ in range(w.outer_loops if loops is None else loops):
        bands, lo, hi = l96_linearise(w, traj)
        prob = Problem(w.s, w.N, w.p, mdl.BandedModel(bands, lo, hi), np.asarray(dr.obs_idx), B, Q, R)
        rhs = l96_rhs(w, prob, obs, traj)
        res = solve_inner(prob, rhs, popts, krylov_kind, tol, maxit)
        dx = prob.split(res.x)[2]
        traj = traj + dx
        trajs.append(traj.copy())
        results.append(res)
    return trajs, results, obs
