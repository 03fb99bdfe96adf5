"""Pins of the oracle's per-time observation blocks (distinct H_i and R_i,
Sec. 2.1's general form): the shared case as a special case, the dense
structure, the primal minimiser, and the spectral statements that do not
depend on H and R being the same at every time."""
import os
import sys

import numpy as np
import pytest
import scipy.linalg as sla

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2105_06975_gb300 import workload as W  # noqa: E402
from oracle import bounds, krylov, model as mdl, problem as prb, saddle as sd  # noqa: E402


def per_time(s=24, N=3, p=8, seed=0):
    w = W.small(W.SCALE, s=s, N=N, p=p).with_(obs_per_time=True)
    dr = W.draws(w, seed)
    return w, dr


def test_draws_per_time_sets_and_other_draws_unchanged():
    w, dr = per_time(s=40, N=4, p=10)
    sets = dr.extra["obs_list"]
    assert len(sets) == w.N + 1
    for o in sets:
        assert len(o) == w.p and np.all(np.diff(o) > 0) and o[0] >= 0 and o[-1] < w.s
    assert any(not np.array_equal(sets[0], o) for o in sets[1:])
    d0 = W.draws(w.with_(obs_per_time=False), 0)
    for name in ("obs_idx", "z_b", "z_q", "z_r", "rhs_probe"):
        assert np.array_equal(getattr(dr, name), getattr(d0, name))


def test_shared_sets_reduce_to_the_shared_problem():
    """With every H_i = H and R_i = R the per-time operators are the shared ones."""
    w, dr = per_time()
    shared = prb.linear_problem(w.with_(obs_per_time=False), W.draws(w.with_(obs_per_time=False), 0))
    pt = sd.PerTimeProblem(w.s, w.N, shared.model, [shared.obs_idx] * (w.N + 1), shared.B, shared.Q,
                           [shared.R] * (w.N + 1))
    assert pt.n == shared.n
    assert np.array_equal(pt.A_dense(), shared.A_dense())
    v = np.random.default_rng(3).standard_normal(pt.n)
    assert np.allclose(pt.A_apply(v), shared.A_apply(v), rtol=0, atol=1e-14)
    assert np.array_equal(pt.join(*pt.split(v)), v)
    for kind, rhat in [("PD", "exact"), ("PI", "rr"), ("PD", "me"), ("PI", "diag")]:
        o = sd.PrecondOptions(kind=kind, k=2, rhat=rhat, kappa_max=10.0)
        a = sd.PerTimePreconditioner(pt, o).apply(v)
        b = sd.Preconditioner(shared, o).apply(v)
        assert np.allclose(a, b, rtol=0, atol=1e-13 * np.linalg.norm(b))


def test_dense_blocks_follow_the_sets():
    w, dr = per_time(s=20, N=2, p=5)
    prob, obs, rhs = prb.per_time_case(w, dr)
    H = prob.H_dense()
    T = w.N + 1
    assert H.shape == (prob.p, w.s * T)
    row = 0
    for i, o in enumerate(dr.extra["obs_list"]):
        for j, col in enumerate(o):
            want = np.zeros(w.s * T)
            want[i * w.s + col] = 1.0
            assert np.array_equal(H[row], want)
            row += 1
    R = prob.R_dense()
    off = 0
    for Ri in prob.R_list:
        m = Ri.shape[0]
        assert np.array_equal(R[off:off + m, off:off + m], Ri)
        assert np.all(R[off:off + m, off + m:] == 0)
        off += m
    # R_i is the SOAR over that time's points: distances from the chord
    o = dr.extra["obs_list"][1]
    r = np.sin(np.pi * abs(o[0] - o[1]) / w.s) / np.pi
    s2, ell = w.soar_r
    assert prob.R_list[1][0, 1] == pytest.approx(s2 * (1 + r / ell) * np.exp(-r / ell), rel=1e-13)
    A = prob.A_dense()
    assert np.array_equal(A, A.T)
    # the matrix-free applies are the dense blocks
    v = np.random.default_rng(8).standard_normal(prob.n)
    assert np.allclose(prob.A_apply(v), A @ v, rtol=0, atol=1e-13 * np.linalg.norm(A @ v))
    for kind in ("PD", "PI"):
        P = sd.PerTimePreconditioner(prob, sd.PrecondOptions(kind=kind, k=2, rhat="me", kappa_max=10.0))
        want = np.linalg.solve(P.dense(), v)
        assert np.allclose(P.apply(v), want, rtol=0, atol=1e-10 * np.linalg.norm(want))


def test_lu_equals_primal_minimiser():
    w, dr = per_time(s=24, N=3, p=8)
    prob, obs, rhs = prb.per_time_case(w, dr)
    g = np.random.default_rng(5)
    rhs = rhs + np.concatenate([g.standard_normal(w.s * (w.N + 1)), np.zeros(prob.n - w.s * (w.N + 1))])
    x_lu = sd.dense_solve(prob, rhs)
    b, d, _ = prob.split(rhs)
    d = np.concatenate(d)
    x_pr = sd.primal_solve(prob, b.ravel(), d)
    assert np.linalg.norm(x_lu - x_pr) <= 1e-9 * np.linalg.norm(x_lu)
    dx = prob.split(x_lu)[2].ravel()
    J0 = sd.linearised_cost(prob, b.ravel(), d, dx)
    for _ in range(3):
        e = g.standard_normal(dx.size)
        assert sd.linearised_cost(prob, b.ravel(), d, dx + 1e-4 * e) >= J0 - 1e-9 * abs(J0)


def test_exact_blocks_mgw_and_schur_pairing():
    """Shat = S: eig = {1, (1 +- sqrt5)/2}; with Dhat = D, Rhat_i = R_i and the
    paper's Shat the non-unit eigenvalues are (1 +- sqrt(1 + 4 mu))/2."""
    w, dr = per_time(s=10, N=3, p=4)
    prob, obs, rhs = prb.per_time_case(w, dr)
    P = sd.PerTimePreconditioner(prob, sd.PrecondOptions(kind="PD", shat="exact"))
    ev = sla.eigvals(prob.A_dense(), P.dense())
    targets = np.array([1.0, (1 + 5 ** 0.5) / 2, (1 - 5 ** 0.5) / 2])
    assert np.min(np.abs(ev.real[:, None] - targets[None, :]), axis=1).max() < 1e-7
    P = sd.PerTimePreconditioner(prob, sd.PrecondOptions(kind="PD", k=2))
    ev = np.sort(sla.eigvals(prob.A_dense(), P.dense()).real)
    mu = sla.eigvals(prob.S_dense(), P.Shat_dense()).real
    pred = np.concatenate([(1 + np.sqrt(1 + 4 * mu)) / 2, (1 - np.sqrt(1 + 4 * mu)) / 2, np.ones(prob.p)])
    assert np.allclose(ev, np.sort(pred), rtol=1e-6, atol=1e-8)


@pytest.mark.parametrize("rhat", ["rr", "diag"])
def test_theorem1_intervals_with_per_time_rhat(rhat):
    w, dr = per_time(s=10, N=3, p=4, seed=2)
    prob, obs, rhs = prb.per_time_case(w, dr)
    P = sd.PerTimePreconditioner(prob, sd.PrecondOptions(kind="PD", k=2, rhat=rhat, kappa_max=5.0))
    ev = sla.eigvals(prob.A_dense(), P.dense())
    assert np.max(np.abs(ev.imag)) < 1e-8
    ext = lambda X, Y: (lambda e: (e[0], e[-1]))(np.sort(sla.eigvalsh(X, Y)))
    D = prob.D_dense()
    lD, LD = ext(D, P.Dhat_dense())
    lR, LR = ext(prob.R_dense(), P.Rhat_dense())
    L = mdl.L_dense(prob.model)
    lS, LS = ext(prob.S_dense(), L.T @ np.linalg.solve(D, L))
    Lh = P.Lhat_dense()
    lL, LL = ext(L.T @ L, Lh.T @ Lh)
    iv = bounds.theorem1_intervals(lD, LD, lR, LR, lS, LS, lL, LL, np.linalg.cond(D))
    assert bounds.in_intervals(ev.real, iv).all()


def test_krylov_solves_reach_lu():
    w, dr = per_time(s=24, N=3, p=8, seed=1)
    prob, obs, rhs = prb.per_time_case(w, dr)
    x_lu = sd.dense_solve(prob, rhs)
    for kind, solver in [("PI", krylov.gmres), ("PD", krylov.minres)]:
        P = sd.PerTimePreconditioner(prob, sd.PrecondOptions(kind=kind, k=2))
        res = solver(prob.A_apply, P.apply, rhs, tol=1e-11, maxit=1000)
        assert res.converged
        assert np.linalg.norm(res.x - x_lu) <= 1e-6 * np.linalg.norm(x_lu)
