"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms
(circulant spectra, Propositions 3 and 4, the Murphy-Golub-Wathen eigenvalues),
structural statements (Lemmas 1 and 2, Propositions 1 and 2, Theorem 1,
Remark 1), independent library routines applied to the assembled matrices
(LU, dense inverses, generalised eigenvalues), brute force on tiny inputs and
relations between numbers the paper prints (Tables 3, 4, 5).
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

from paper_2105_06975_gb300 import workload as W
from oracle import bounds, covariance as cov, krylov, model as mdl, problem as prb, saddle as sd

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def tiny(s=12, N=4, p=6, seed=0, obs="even"):
    w = W.small(W.TINY, s=s, N=N, p=p).with_(obs=obs)
    return w, W.draws(w, seed)


def random_banded(s, N, lo, hi, seed, scale=0.4):
    g = np.random.default_rng(seed)
    return mdl.BandedModel(scale * g.standard_normal((N, s, lo + hi + 1)), lo, hi)


def rand_problem(s=8, N=4, p=4, seed=1, model=None, spd_scale=1.0):
    """A generic small problem: random SPD B, Q, R and random banded M."""
    g = np.random.default_rng(seed)

    def spd(m):
        X = g.standard_normal((m, m))
        return spd_scale * (X @ X.T / m + 0.3 * np.eye(m))
    obs = np.sort(g.choice(s, p, replace=False))
    model = model or random_banded(s, N, 1, 1, seed + 7)
    return sd.Problem(s, N, p, model, obs, spd(s), spd(s), spd(p))


# ------------------------------------------------------------ covariances
def test_soar_circulant_spectrum_closed_form():
    """B on the periodic grid is circulant (Sec. 6.1): its eigenvalues are the
    DFT of its first row."""
    for s, (s2, ell) in [(64, (1.0, 0.1)), (100, (0.05, 0.05)), (37, (0.5, 0.2))]:
        B = cov.soar_state(s, s2, ell)
        ev = np.sort(np.linalg.eigvalsh(B))
        dft = np.sort(np.real(np.fft.fft(B[0])))
        assert np.allclose(ev, dft, rtol=0, atol=1e-12 * ev[-1])
        assert np.allclose(B, B.T)
        assert ev[0] > 0


def test_soar_entries_from_geometry():
    """Entries against chord lengths of a circle of circumference 1: opposite
    points are a diameter 1/pi apart, quarter-circle points sqrt(2)/(2 pi)."""
    s, s2, ell = 16, 0.7, 0.15
    B = cov.soar_state(s, s2, ell)
    c = lambda r: s2 * (1 + r / ell) * math.exp(-r / ell)
    assert B[0, 0] == pytest.approx(s2, rel=1e-15)
    assert B[0, 8] == pytest.approx(c(1 / math.pi), rel=1e-14)
    assert B[3, 7] == pytest.approx(c(math.sqrt(2) / (2 * math.pi)), rel=1e-14)
    # R over observed points uses the same function at those positions
    R = cov.soar_obs(s, np.array([0, 4, 8]), s2, ell)
    assert R[0, 2] == pytest.approx(c(1 / math.pi), rel=1e-14)


def test_ridge_regression_prop3():
    """Prop. 3: eig(R_RR^{-1} R) = lambda/(lambda+gamma); kappa(R_RR) = kappa_max."""
    w, dr = tiny(s=40, N=2, p=20)
    R = cov.soar_obs(w.s, dr.obs_idx, 0.1, 0.2)
    lam = np.linalg.eigvalsh(R)
    assert lam[-1] / lam[0] > 100
    Rrr, gamma = cov.r_ridge(R, 100.0)
    assert gamma == pytest.approx((lam[-1] - 100 * lam[0]) / 99, rel=1e-10)
    got = np.sort(sla.eigh(R, Rrr, eigvals_only=True))
    want = np.sort(lam / (lam + gamma))
    assert np.allclose(got, want, rtol=1e-9, atol=1e-12)
    lr = np.linalg.eigvalsh(Rrr)
    assert lr[-1] / lr[0] == pytest.approx(100.0, rel=1e-9)
    # already better conditioned than kappa_max: no shift
    assert cov.r_ridge(np.diag([1.0, 2.0, 3.0]), 100.0)[1] == 0.0


def test_min_eigenvalue_prop4():
    """Prop. 4: eig(R_ME^{-1} R) = 1 above T, lambda/T at or below T."""
    w, dr = tiny(s=40, N=2, p=20)
    R = cov.soar_obs(w.s, dr.obs_idx, 0.1, 0.2)
    lam = np.linalg.eigvalsh(R)
    Rme, T = cov.r_min_eig(R, 100.0)
    assert T == pytest.approx(lam[-1] / 100, rel=1e-14)
    got = np.sort(sla.eigh(R, Rme, eigvals_only=True))
    want = np.sort(np.where(lam > T, 1.0, lam / T))
    assert np.allclose(got, want, rtol=1e-9, atol=1e-12)
    lm = np.linalg.eigvalsh(Rme)
    assert lm[-1] / lm[0] == pytest.approx(100.0, rel=1e-9)
    assert np.allclose(Rme, Rme.T, atol=1e-14)


# ------------------------------------------------------------------ model
def test_advdiff_step_is_contraction_with_unit_norm():
    """Upwind advection + diffusion: rows sum to 1 (mass conserved) and the
    circulant symbol has modulus at most 1, attained at zero frequency."""
    m = mdl.StencilModel(32, 3, mdl.advdiff_coeffs(0.5, 0.2))
    M = m.dense(1)
    assert np.allclose(M.sum(axis=1), 1.0)
    assert np.linalg.norm(M, 2) == pytest.approx(1.0, abs=1e-12)
    assert mdl.advdiff_coeffs(0.5, 0.2) == pytest.approx((0.7, 0.1, 0.2))
    x = np.random.default_rng(0).standard_normal(32)
    y = np.random.default_rng(1).standard_normal(32)
    assert m.apply(1, x) @ y == pytest.approx(x @ m.apply_T(1, y), rel=1e-13)
    assert np.allclose(m.apply(1, x), M @ x)


@pytest.mark.parametrize("k", [1, 2, 3, 5, 6])
def test_lemma1_blocks_and_sweeps(k):
    """Lemma 1 block formula == dense inverse of L_M(k) == the sweep recursion."""
    s, N = 5, 5
    m = random_banded(s, N, 2, 1, seed=k)
    LM = mdl.LM_dense(m, k)
    inv = np.linalg.inv(LM)
    for i in range(1, N + 2):
        for j in range(1, N + 2):
            blk = inv[(i - 1) * s:i * s, (j - 1) * s:j * s]
            assert np.allclose(blk, mdl.lemma1_block(m, k, i, j), atol=1e-12)
    v = np.random.default_rng(k).standard_normal((N + 1, s))
    assert np.allclose(mdl.LM_inv(m, v, k).ravel(), inv @ v.ravel(), atol=1e-12)
    assert np.allclose(mdl.LM_inv_T(m, v, k).ravel(), inv.T @ v.ravel(), atol=1e-12)
    assert np.allclose(mdl.LM_apply(m, v, k).ravel(), LM @ v.ravel(), atol=1e-13)


def test_lm_special_cases():
    """L_M(1) = L_0 = I (Sec. 2.2) and L_M(N+1) = L (after Lemma 1)."""
    s, N = 4, 6
    m = random_banded(s, N, 1, 1, seed=3)
    assert np.array_equal(mdl.LM_dense(m, 1), np.eye((N + 1) * s))
    L = np.eye((N + 1) * s)
    for t in range(1, N + 1):
        L[t * s:(t + 1) * s, (t - 1) * s:t * s] = -m.dense(t)
    assert np.array_equal(mdl.LM_dense(m, N + 1), L)
    v = np.random.default_rng(0).standard_normal((N + 1, s))
    assert np.allclose(mdl.L_apply(m, v).ravel(), L @ v.ravel())
    assert np.allclose(mdl.LT_apply(m, v).ravel(), L.T @ v.ravel())


@pytest.mark.parametrize("N,k", [(6, 2), (7, 3), (8, 4), (5, 5)])
def test_lemma2_structure(N, k):
    """Lemma 2: L_M^{-T} L^T L L_M^{-1} - I has, for n = 1..floor(N/k), the
    blocks (M_nk..M_i)^T (M_nk..M_j) on chunk n and -(M_nk..M_j) on row nk+1
    (1-based block indices), zero elsewhere."""
    s = 3
    m = random_banded(s, N, 1, 1, seed=N * 10 + k)
    L = mdl.L_dense(m)
    LMi = np.linalg.inv(mdl.LM_dense(m, k))
    Amat = LMi.T @ L.T @ L @ LMi - np.eye((N + 1) * s)

    def chain(top, low):   # M_top M_{top-1} ... M_low (1-based model indices)
        P = np.eye(s)
        for t in range(top, low - 1, -1):
            P = P @ m.dense(t)
        return P
    want = np.zeros_like(Amat)

    def put(i, j, blk):
        want[(i - 1) * s:i * s, (j - 1) * s:j * s] += blk
    for n in range(1, N // k + 1):
        lo_, hi_ = (n - 1) * k + 1, n * k
        for i in range(lo_, hi_ + 1):
            for j in range(lo_, hi_ + 1):
                put(i, j, chain(n * k, i).T @ chain(n * k, j))
            put(n * k + 1, i, -chain(n * k, i))
            put(i, n * k + 1, -chain(n * k, i).T)
    assert np.allclose(Amat, want, atol=1e-11)


@pytest.mark.parametrize("N,k", [(5, 2), (5, 3), (6, 3), (6, 4), (7, 8), (9, 4)])
def test_prop1_unit_eigenvalues(N, k):
    """Prop. 1: at least (N+1-2 floor(N/k)) s unit eigenvalues."""
    s = 4
    m = random_banded(s, N, 1, 2, seed=100 + N * k, scale=0.6)
    L = mdl.L_dense(m)
    LMi = np.linalg.inv(mdl.LM_dense(m, k))
    ev = np.linalg.eigvalsh(LMi.T @ L.T @ L @ LMi)
    n_unit = int(np.sum(np.abs(ev - 1.0) < 1e-8))
    assert n_unit >= bounds.prop1_unit_count(N, k, s)


@pytest.mark.parametrize("N,k", [(6, 2), (6, 3), (8, 3), (5, 4), (7, 7)])
def test_prop2_upper_bound(N, k):
    """Prop. 2 / Remark 3 with ||M M^T|| <= 1: the advection-diffusion step
    and random contractions."""
    s = 6
    for m in (mdl.StencilModel(s, N, mdl.advdiff_coeffs(0.5, 0.2)),
              random_banded(s, N, 1, 1, seed=N + k)):
        if isinstance(m, mdl.BandedModel):
            for t in range(1, N + 1):
                nrm = np.linalg.norm(m.dense(t), 2)
                m.bands[t - 1] /= nrm
                m._csr.clear()
        L = mdl.L_dense(m)
        LMi = np.linalg.inv(mdl.LM_dense(m, k))
        lmax = np.linalg.eigvalsh(LMi.T @ L.T @ L @ LMi)[-1]
        assert lmax <= bounds.prop2_upper(N, k) + 1e-10


# ---------------------------------------------------- saddle-point system
def test_structured_applies_match_dense_definitions():
    """Sec. 6.2 blockwise applies == the assembled matrices of Eq. saddlepointA
    and Eq. prec (dense solves), for P_D and P_I over k and Rhat choices."""
    w, dr = tiny(s=10, N=4, p=5)
    prob = prb.linear_problem(w, dr)
    A = prob.A_dense()
    assert np.array_equal(A, A.T)
    v = np.random.default_rng(0).standard_normal(prob.n)
    assert np.allclose(prob.A_apply(v), A @ v, rtol=0, atol=1e-12 * np.abs(A).sum(1).max())
    for kind in ("PD", "PI"):
        for k in (1, 2, 5):
            for rh in ("exact", "rr", "me", "diag"):
                P = sd.Preconditioner(prob, sd.PrecondOptions(kind=kind, k=k, rhat=rh))
                Pd = P.dense()
                got = P.apply(v)
                want = np.linalg.solve(Pd, v)
                assert np.linalg.norm(got - want) <= 1e-8 * np.linalg.norm(want), (kind, k, rh)
                if kind == "PD":
                    np.linalg.cholesky(Pd)          # P_D is SPD (Sec. 3)


def test_dense_lu_equals_primal_minimiser():
    """O1 vs O2: LU of the saddle-point matrix == the normal-equations
    minimiser of the linearised cost; the cost is stationary there."""
    w, dr = tiny(s=20, N=4, p=10)
    prob, obs, rhs = prb.linear_case(w, dr)
    rng = np.random.default_rng(5)
    rhs = rhs + np.concatenate([rng.standard_normal(prob.s * (prob.N + 1)), np.zeros(prob.n - prob.s * (prob.N + 1))])
    x_lu = sd.dense_solve(prob, rhs)
    b, d, _ = prob.split(rhs)
    x_pr = sd.primal_solve(prob, b.ravel(), d.ravel())
    assert np.linalg.norm(x_lu - x_pr) <= 1e-9 * np.linalg.norm(x_lu)
    dx = prob.split(x_lu)[2].ravel()
    J0 = sd.linearised_cost(prob, b.ravel(), d.ravel(), dx)
    for _ in range(3):
        e = rng.standard_normal(dx.size)
        for eps in (1e-3, 1e-5):
            assert sd.linearised_cost(prob, b.ravel(), d.ravel(), dx + eps * e) >= J0 - 1e-9 * abs(J0)


def test_mgw_exact_blocks_three_eigenvalues():
    """With Dhat = D, Rhat = R and Shat = S, eig(P_D^{-1} A) = {1, (1 +- sqrt5)/2}
    (Murphy-Golub-Wathen, cited in Sec. 2.1) and MINRES stops within 3 steps."""
    w, dr = tiny(s=12, N=3, p=6)
    prob, obs, rhs = prb.linear_case(w, dr)
    P = sd.Preconditioner(prob, sd.PrecondOptions(kind="PD", shat="exact"))
    ev = sla.eigvals(prob.A_dense(), P.dense())
    assert np.max(np.abs(ev.imag)) < 1e-8
    targets = np.array([1.0, (1 + 5 ** 0.5) / 2, (1 - 5 ** 0.5) / 2])
    dist = np.min(np.abs(ev.real[:, None] - targets[None, :]), axis=1)
    assert dist.max() < 1e-7
    res = krylov.minres(prob.A_apply, P.apply, rhs, tol=1e-10)
    assert res.iters <= 3 or res.iters <= 5 and res.relres_true < 1e-10
    assert res.relres_true < 1e-9


def test_schur_pairing_and_table3_relation():
    """With Dhat = D and Rhat = R the non-unit eigenvalues of P_D^{-1} A are
    (1 +- sqrt(1 + 4 mu))/2, mu in eig(Shat^{-1} S), so they pair as lambda and
    1 - lambda.  The paper's Table 3 rows with Rhat = R show the same pairing
    (-3.6119 + 4.6119 = 1, -2.0415 + 3.0415 = 1) and min positive eigenvalue 1."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table3_eigs.txt")) if l.strip() and not l.startswith("#")]
    for Lh, Rh, lmin, maxneg, minpos, lmax in rows:
        if Rh == "R":
            assert float(lmin) + float(lmax) == pytest.approx(1.0, abs=1e-4)
            assert float(minpos) == pytest.approx(1.0, abs=1e-4)
    w, dr = tiny(s=10, N=4, p=5)
    prob = prb.linear_problem(w, dr)
    for k in (1, 3):
        P = sd.Preconditioner(prob, sd.PrecondOptions(kind="PD", k=k))
        ev = np.sort(sla.eigvals(prob.A_dense(), P.dense()).real)
        mu = sla.eigvals(prob.S_dense(), P.Shat_dense()).real
        pred = np.concatenate([(1 + np.sqrt(1 + 4 * mu)) / 2, (1 - np.sqrt(1 + 4 * mu)) / 2,
                               np.ones(prob.p * (prob.N + 1))])
        assert np.allclose(ev, np.sort(pred), rtol=1e-6, atol=1e-8)
        assert ev[0] + ev[-1] == pytest.approx(1.0, abs=1e-8)


@pytest.mark.parametrize("k,rhat,dhat", [(1, "exact", "exact"), (3, "rr", "exact"), (2, "me", "rr"),
                                         (4, "diag", "exact"), (5, "rr", "rr")])
def test_theorem1_intervals_contain_spectrum(k, rhat, dhat):
    """Theorem 1: eig(P_D^{-1} A) lies in the three stated intervals."""
    prob = rand_problem(s=6, N=4, p=3, seed=k)
    P = sd.Preconditioner(prob, sd.PrecondOptions(kind="PD", k=k, rhat=rhat, dhat=dhat, kappa_max=3.0))
    ev = sla.eigvals(prob.A_dense(), P.dense())
    assert np.max(np.abs(ev.imag)) < 1e-8
    ext = lambda X, Y: (lambda e: (e[0], e[-1]))(np.sort(sla.eigvalsh(X, Y)))
    D = prob.D_dense()
    lD, LD = ext(D, P.Dhat_dense())
    lR, LR = ext(prob.R_dense(), np.kron(np.eye(prob.N + 1), P.Rhat))
    L = mdl.L_dense(prob.model)
    St = L.T @ np.linalg.solve(D, L)
    lS, LS = ext(prob.S_dense(), St)
    Lh = P.Lhat_dense()
    lL, LL = ext(L.T @ L, Lh.T @ Lh)
    kD = np.linalg.cond(D)
    iv = bounds.theorem1_intervals(lD, LD, lR, LR, lS, LS, lL, LL, kD)
    assert bounds.in_intervals(ev.real, iv).all()


def test_r_diag_is_the_diagonal():
    """Sec. 5.1: R_diag keeps R's diagonal only.  A SOAR R has the constant
    diagonal sigma^2, so R_diag = sigma^2 I and eig(R_diag^{-1} R) = eig(R)/sigma^2."""
    w, dr = tiny(s=40, N=2, p=20)
    R = cov.soar_obs(w.s, dr.obs_idx, 0.1, 0.2)
    Rd = cov.r_diag(R)
    assert np.array_equal(Rd, 0.1 * np.eye(R.shape[0]))
    assert np.array_equal(cov.rhat(R, "diag"), Rd)
    got = np.sort(sla.eigh(R, Rd, eigvals_only=True))
    assert np.allclose(got, np.linalg.eigvalsh(R) / 0.1, rtol=1e-12)
    M = np.array([[4.0, 1.0, 2.0], [1.0, 3.0, 0.5], [2.0, 0.5, 5.0]])
    assert np.array_equal(cov.r_diag(M), np.diag([4.0, 3.0, 5.0]))


def test_bd_intervals_attained_on_decoupled_blocks():
    """Eq. BDPrecBounds against saddle points small enough to solve by hand.
    One block each (Phi = [a], B = [b], preconditioner diag(ah, sh)):
    eig = roots of lambda^2 - d lambda - d mu (d = a/ah, mu = (b^2/a)/sh),
    and with delta = Delta = d, phi = Phi = mu all four outer ends are those
    roots.  Phi = diag(a1, a2) with B = [b, 0]: the eigenvalues are d2 and the
    roots for d1; the positive root is the positive interval's lower end when
    d1 is the smaller ratio and its upper end when d1 is the larger.  Exact
    blocks give the MGW values."""
    for a, ah, b, sh in [(2.0, 4.0, 1.3, 0.7), (5.0, 2.0, 0.4, 2.5)]:
        ev = np.sort(sla.eigvals(np.array([[a, b], [b, 0.0]]), np.diag([ah, sh])).real)
        d, mu = a / ah, b * b / a / sh
        lm, lp = (d - math.sqrt(d * d + 4 * d * mu)) / 2, (d + math.sqrt(d * d + 4 * d * mu)) / 2
        assert np.allclose(ev, [lm, lp], rtol=1e-12)
        neg, mid, pos = bounds.bd_intervals(d, d, mu, mu)
        assert neg == pytest.approx((lm, lm), rel=1e-12) and pos == pytest.approx((lp, lp), rel=1e-12)
        assert mid == (d, d)
    for a1, a2, a1h, a2h, b, sh in [(2.0, 3.0, 4.0, 1.5, 1.3, 0.7), (5.0, 1.0, 2.0, 4.0, 0.4, 2.5)]:
        A = np.array([[a1, 0, b], [0, a2, 0], [b, 0, 0]])
        ev = np.sort(sla.eigvals(A, np.diag([a1h, a2h, sh])).real)
        d1, d2 = a1 / a1h, a2 / a2h
        mu = b * b / a1 / sh
        lm, lp = (d1 - math.sqrt(d1 * d1 + 4 * d1 * mu)) / 2, (d1 + math.sqrt(d1 * d1 + 4 * d1 * mu)) / 2
        assert np.allclose(ev, np.sort([lm, d2, lp]), rtol=1e-12)
        neg, mid, pos = bounds.bd_intervals(min(d1, d2), max(d1, d2), mu, mu)
        assert bounds.in_intervals(ev, (neg, mid, pos), rtol=1e-12).all()
        assert neg[0] <= lm <= neg[1] and mid[0] <= d2 <= mid[1]
        assert lp == pytest.approx(pos[0] if d1 < d2 else pos[1], rel=1e-12)
    mgw = bounds.bd_intervals(1.0, 1.0, 1.0, 1.0)
    for (lo, hi), v in zip(mgw, [(1 - 5 ** 0.5) / 2, 1.0, (1 + 5 ** 0.5) / 2]):
        assert lo == pytest.approx(v, rel=1e-15) and hi == pytest.approx(v, rel=1e-15)


def test_remark1_symmetric_closed_form_and_iteration_count():
    """For [-b, -a] U [a, b] the factor per two MINRES steps is the
    Chebyshev one on [a^2, b^2]: (b - a)/(b + a).  Unequal widths are
    stretched to the wider one, which can only raise the factor.  The
    iteration count is the smallest even 2l with 2 rho^l <= tol."""
    for a, b in [(0.5, 2.0), (1.0, 1.0), (1e-3, 10.0)]:
        assert bounds.remark1_factor(b, a, a, b) == pytest.approx((b - a) / (b + a), rel=1e-14, abs=1e-15)
    r_un = bounds.remark1_factor(3.0, 1.0, 0.5, 1.0)           # widths 2 and 0.5
    assert r_un == pytest.approx(bounds.remark1_factor(3.0, 1.0, 0.5, 2.5), rel=1e-15)
    assert r_un > bounds.remark1_factor(1.5, 1.0, 0.5, 1.0)
    for mus, tol in [((2.0, 0.5, 0.5, 2.0), 1e-6), ((4.0, 0.3, 0.7, 3.1), 1e-8), ((1.0, 0.9, 0.9, 1.0), 1e-3)]:
        rho = bounds.remark1_factor(*mus)
        it = bounds.remark1_iterations(*mus, tol)
        l = it // 2
        assert it % 2 == 0 and 2 * rho ** l <= tol * (1 + 1e-12)
        assert l == 1 or 2 * rho ** (l - 1) > tol


def test_remark1_minres_rate():
    """Remark 1: ||r_2l||_{P^{-1}} <= 2 rho^l ||r_0||_{P^{-1}} with rho from the
    computed eigenvalue intervals; the oracle's |eta| is that norm."""
    prob = rand_problem(s=8, N=4, p=4, seed=11)
    P = sd.Preconditioner(prob, sd.PrecondOptions(kind="PD", k=2, rhat="rr", kappa_max=4.0))
    ev = np.sort(sla.eigvals(prob.A_dense(), P.dense()).real)
    neg, pos = ev[ev < 0], ev[ev > 0]
    rho = bounds.remark1_factor(-neg[0], -neg[-1], pos[0], pos[-1])
    b = np.random.default_rng(2).standard_normal(prob.n)
    res = krylov.minres(prob.A_apply, P.apply, b, tol=1e-12, maxit=200, check_true=False)
    for j, h in enumerate(res.history, start=1):
        if j % 2 == 0:
            assert h <= 2 * rho ** (j // 2) * (1 + 1e-8) + 1e-13


def test_minres_eta_is_preconditioned_residual_norm():
    prob = rand_problem(s=8, N=3, p=4, seed=4)
    P = sd.Preconditioner(prob, sd.PrecondOptions(kind="PD", k=2))
    Pd = P.dense()
    b = np.random.default_rng(3).standard_normal(prob.n)
    nrm = lambda r: math.sqrt(r @ np.linalg.solve(Pd, r))
    r0 = nrm(b)
    for j in (1, 2, 5, 9):
        res = krylov.minres(prob.A_apply, P.apply, b, tol=0.0, maxit=j, check_true=False)
        assert res.history[-1] * r0 == pytest.approx(nrm(b - prob.A_apply(res.x)), rel=1e-8)


def test_gmres_recurrence_is_true_residual_and_finite_termination():
    prob = rand_problem(s=6, N=3, p=3, seed=9)
    P = sd.Preconditioner(prob, sd.PrecondOptions(kind="PI", k=2))
    b = np.random.default_rng(1).standard_normal(prob.n)
    nb = np.linalg.norm(b)
    for j in (1, 3, 7):
        res = krylov.gmres(prob.A_apply, P.apply, b, tol=0.0, maxit=j)
        assert res.history[-1] == pytest.approx(np.linalg.norm(b - prob.A_apply(res.x)) / nb, rel=1e-7)
    res = krylov.gmres(prob.A_apply, P.apply, b, tol=1e-12, maxit=prob.n)
    assert res.converged and res.iters <= prob.n
    assert np.allclose(res.x, np.linalg.solve(prob.A_dense(), b), rtol=1e-7, atol=1e-9)


def test_krylov_solutions_match_lu():
    w, dr = tiny(s=24, N=5, p=12)
    prob, obs, rhs = prb.linear_case(w, dr)
    x_lu = sd.dense_solve(prob, rhs)
    for popts, kk in [(sd.PrecondOptions(kind="PD", k=3), "minres"),
                      (sd.PrecondOptions(kind="PI", k=3, rhat="rr"), "gmres")]:
        res = prb.solve_inner(prob, rhs, popts, kk, tol=1e-10, maxit=2000)
        assert res.converged
        assert np.linalg.norm(res.x - x_lu) <= 1e-5 * np.linalg.norm(x_lu)
    # flexible GMRES with a fixed preconditioner == GMRES
    P = sd.Preconditioner(prob, sd.PrecondOptions(kind="PI", k=2))
    r1 = krylov.gmres(prob.A_apply, P.apply, rhs, tol=1e-8)
    r2 = krylov.gmres(prob.A_apply, lambda v, j: P.apply(v), rhs, tol=1e-8, flexible=True)
    assert r1.iters == r2.iters and np.allclose(r1.x, r2.x)


def test_product_counts_tables_4_5():
    """Counting convention of Tables 4 and 5: per iteration P_D costs (N+1)
    R_i, 2(N+1) D_i and (N+1) Dhat_i^{-1} products; P_I costs (N+1) R_i and
    2(N+1) D_i.  The printed totals obey these ratios with N+1 = 16."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table4_5_counts.txt")) if l.strip() and not l.startswith("#")]
    for tab, kind, rh, k, Ri, Rhi, Di, Dhi in rows:
        Ri, Rhi, Di, Dhi = int(Ri), int(Rhi), int(Di), int(Dhi)
        assert Ri % 16 == 0 and Di == 2 * Ri
        if Rhi >= 0:
            assert Rhi == Ri
        if kind == "PD":
            assert Dhi == Ri
    # the oracle's solvers make exactly these products per iteration
    w, dr = tiny(s=10, N=3, p=5)
    for kind, kk in (("PD", "minres"), ("PI", "gmres")):
        prob, obs, rhs = prb.linear_case(w, dr)
        cnt = {"D": 0, "R": 0, "Dh": 0, "Rh": 0}
        P = sd.Preconditioner(prob, sd.PrecondOptions(kind=kind, k=2))

        def wrap(obj, name, key, per):
            f = getattr(obj, name)
            def g(*a):
                cnt[key] += per
                return f(*a)
            setattr(obj, name, g)
        wrap(prob, "D_apply", "D", prob.N + 1)
        wrap(prob, "R_apply", "R", prob.N + 1)
        wrap(P, "Dhat_inv", "Dh", prob.N + 1)
        wrap(P, "Rhat_inv", "Rh", prob.N + 1)
        fn = krylov.minres if kk == "minres" else krylov.gmres
        res = fn(prob.A_apply, P.apply, rhs, tol=0.0, maxit=7, **({"check_true": False} if kk == "minres" else {}))
        # iterations + the initial preconditioner apply (MINRES) / final residual check
        T = prob.N + 1
        if kind == "PD":
            n_prec = 7 + 1
            assert cnt["Dh"] == n_prec * T and cnt["Rh"] == n_prec * T
            assert cnt["D"] == (7 + 1) * T + n_prec * T      # A applies (+ true residual) + Shat
        else:
            assert cnt["Dh"] == 0 and cnt["Rh"] == 7 * T
            assert cnt["D"] == (7 + 2) * T + 7 * T           # A applies (+ r0 + final) + P_I's D c1
        assert cnt["R"] == (8 if kind == "PD" else 9) * T           # one per A apply


# -------------------------------------------------------------- Lorenz-96
def test_l96_fixed_point_and_tlm():
    F, dt = 8.0, 0.025
    x = np.full(80, F)
    assert np.all(mdl.l96_rhs(x, F) == 0.0)
    assert np.array_equal(mdl.rk4_step(x, dt, F), x)
    g = np.random.default_rng(0)
    x = F + g.standard_normal(80)
    v = g.standard_normal(80)
    M = mdl.l96_tlm(x, dt, F, 5)
    base = mdl.l96_forecast(x, dt, F, 5)
    errs = []
    for eps in (1e-2, 1e-3, 1e-4):
        errs.append(np.linalg.norm(mdl.l96_forecast(x + eps * v, dt, F, 5) - base - eps * (M @ v)))
    assert errs[1] / errs[0] < 0.02 and errs[2] / errs[1] < 0.02      # O(eps^2)
    wv = g.standard_normal(80)
    assert (M @ v) @ wv == pytest.approx(v @ (M.T @ wv), rel=1e-13)
    lo, hi = mdl.band_width(5)
    assert (lo, hi) == (40, 20)
    bands = mdl.to_bands(M, lo, hi)          # raises if anything lies outside
    bm = mdl.BandedModel(bands[None], lo, hi)
    assert np.allclose(bm.apply(1, v), M @ v, atol=1e-13)


def test_l96_rhs_hand_evaluated_with_periodic_wrap():
    """Sec. 7.1: dx_j/dt = (x_{j+1} - x_{j-2}) x_{j-1} - x_j + F, periodic.
    On x_j = j + 1 (s = 8, 0-based j) the interior entries are
    (3)(j) - (j+1) + F = 2j + 7, and the wrapped ends are worked out by hand:
      j = 0: (x_1 - x_6) x_7 - x_0 + 8 = (2 - 7) 8 - 1 + 8 = -33
      j = 1: (x_2 - x_7) x_0 - x_1 + 8 = (3 - 8) 1 - 2 + 8 =   1
      j = 7: (x_0 - x_5) x_6 - x_7 + 8 = (1 - 6) 7 - 8 + 8 = -35
    A mirrored stencil (x_{j-1} - x_{j+2}) x_{j+1} or a swapped pair of roll
    offsets changes these values, which the constant fixed point cannot see."""
    x = np.arange(1.0, 9.0)
    f = mdl.l96_rhs(x, 8.0)
    expected = np.array([-33.0, 1.0, 11.0, 13.0, 15.0, 17.0, 19.0, -35.0])
    assert np.array_equal(f, expected)
    # forcing enters additively, once
    assert np.array_equal(mdl.l96_rhs(x, 0.0), expected - 8.0)


def test_rk4_step_is_classical_fourth_order(monkeypatch):
    """The Runge-Kutta scheme of Sec. 7.1 is the classical fourth-order one.
    (i) On the linear test equation dx/dt = lam x one classical RK4 step
    multiplies x by the degree-4 Taylor polynomial of exp(lam dt), exactly (up
    to rounding); a wrong stage weight or stage point breaks that identity.
    (ii) On the Lorenz-96 right-hand side itself, the global error at t = 0.5
    against a fine-step solution falls by 2^4 per halving of dt."""
    lam = np.array([-0.7, 0.3, -2.0, 1.1])
    monkeypatch.setattr(mdl, "l96_rhs", lambda x, F: lam * x)
    x0 = np.array([1.0, -2.0, 0.5, 3.0])
    for dt in (0.1, 0.37):
        z = lam * dt
        taylor = 1.0 + z + z ** 2 / 2.0 + z ** 3 / 6.0 + z ** 4 / 24.0
        np.testing.assert_allclose(mdl.rk4_step(x0, dt, 0.0), taylor * x0, rtol=1e-15, atol=0)
    monkeypatch.undo()

    g = np.random.default_rng(3)
    x = 8.0 + g.standard_normal(40)
    T = 0.5
    ref = mdl.l96_forecast(x, T / 4096, 8.0, 4096)
    errs = [np.linalg.norm(mdl.l96_forecast(x, T / m, 8.0, m) - ref) for m in (32, 64, 128)]
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    for r in ratios:
        assert 13.0 < r < 19.0, ratios


def test_gauss_newton_linear_converges_in_one_loop():
    """For a linear model the first inner solve is the full answer: the second
    outer loop's increment is zero to solver tolerance (Sec. 2.1)."""
    w, dr = tiny(s=16, N=4, p=8)
    prob, obs, rhs = prb.linear_case(w, dr)
    traj = prb.background_trajectory_linear(prob, obs.xb)
    x1 = sd.dense_solve(prob, rhs)
    traj = traj + prob.split(x1)[2]
    rhs2 = prb.rhs_linear(prob, obs, traj)
    x2 = sd.dense_solve(prob, rhs2)
    assert np.linalg.norm(prob.split(x2)[2]) <= 1e-9 * np.linalg.norm(prob.split(x1)[2])


def test_gauss_newton_l96_rhs_and_convergence():
    """C1: the inner right-hand side about x^(l) makes the linearised cost at
    dx = 0 equal the nonlinear cost (Eq. CostFn, no 1/2 factors), and its
    first-order change matches the nonlinear one.  Over the outer loops the
    cost falls and the increments shrink (Sec. 2.1)."""
    w = W.small(W.L96, s=40, N=4, p=20).with_(spinup_steps=200, steps_per_obs=2)
    dr = W.draws(w, 0)
    popts = sd.PrecondOptions(kind="PI", k=3)
    trajs, results, obs = prb.gauss_newton_l96(w, dr, popts, "gmres", tol=1e-10, maxit=2000)
    B, Q, R = prb.covariances(w, dr.obs_idx)

    def J(traj):
        e0 = traj[0] - obs.xb
        out = e0 @ np.linalg.solve(B, e0)
        for t in range(w.N + 1):
            e = obs.y[t] - traj[t, dr.obs_idx]
            out += e @ np.linalg.solve(R, e)
        for t in range(1, w.N + 1):
            e = traj[t] - mdl.l96_forecast(traj[t - 1], w.dt, w.forcing, w.steps_per_obs)
            out += e @ np.linalg.solve(Q, e)
        return out
    costs = [J(t) for t in trajs]
    assert costs[-1] < 0.2 * costs[0]
    assert all(r.converged for r in results)
    inc = [np.linalg.norm(trajs[i + 1] - trajs[i]) for i in range(len(trajs) - 1)]
    assert inc[-1] < 0.1 * inc[0]
    traj = trajs[0]
    bands, lo, hi = prb.l96_linearise(w, traj)
    prob = sd.Problem(w.s, w.N, w.p, mdl.BandedModel(bands, lo, hi), np.asarray(dr.obs_idx), B, Q, R)
    b, d, _ = prob.split(prb.l96_rhs(w, prob, obs, traj))
    zero = np.zeros(prob.s * (prob.N + 1))
    assert sd.linearised_cost(prob, b.ravel(), d.ravel(), zero) == pytest.approx(costs[0], rel=1e-12)
    e = np.random.default_rng(4).standard_normal(zero.size)
    for eps in (1e-4, 1e-5):
        lin = sd.linearised_cost(prob, b.ravel(), d.ravel(), eps * e) - costs[0]
        non = J(traj + eps * e.reshape(traj.shape)) - costs[0]
        assert lin == pytest.approx(non, rel=10 * eps)


# ------------------------------------------------------ learned Schur block
def test_learned_conv_matches_dense_definition():
    """The periodic conv equals the dense matrix built entry by entry from
    out[co, x] = b[co] + sum W[co, ci, k] in[ci, (x + k - 2) mod s]."""
    from oracle import learned as ln
    g = np.random.default_rng(3)
    W = g.standard_normal((4, 3, ln.KW))
    b = g.standard_normal(4)
    x = g.standard_normal((3, 11))
    ref = (ln.conv_matrix(W, 11) @ x.ravel()).reshape(4, 11) + b[:, None]
    assert np.max(np.abs(ln.conv1d(x, W, b) - ref)) < 1e-13


def test_learned_backward_matches_finite_differences():
    """Every weight and bias gradient of |z - t|^2/|t|^2 against central
    differences in FP64 (step 1e-6): relative error below 1e-6."""
    from oracle import learned as ln
    g = np.random.default_rng(4)
    params = ln.init_params(3, 5, seed=7)
    params = [(W + 0.05 * g.standard_normal(W.shape), b + 0.05 * g.standard_normal(b.shape)) for W, b in params]
    y = g.standard_normal((3, 13))
    t = y + 0.3 * g.standard_normal((3, 13))
    _, grads = ln.backward(params, y, t)
    h = 1e-6
    worst = 0.0
    for li in range(4):
        for which in (0, 1):
            arr = params[li][which]
            gref = grads[li][which]
            for idx in np.ndindex(arr.shape):
                old = arr[idx]
                arr[idx] = old + h
                lp = ln.loss(params, y, t)
                arr[idx] = old - h
                lm = ln.loss(params, y, t)
                arr[idx] = old
                fd = (lp - lm) / (2 * h)
                worst = max(worst, abs(fd - gref[idx]) / max(1e-8, abs(fd) + abs(gref[idx])))
    assert worst < 1e-6, worst


def test_learned_preconditioner_is_scale_equivariant():
    """z(alpha y) = alpha z(y) for alpha > 0: the input is normalised before the
    network and the output rescaled, so the preconditioner commutes with the
    residual's scale (as a Krylov preconditioner must, up to rounding)."""
    from oracle import learned as ln
    g = np.random.default_rng(5)
    params = ln.init_params(3, 4, seed=2)
    y = g.standard_normal((3, 9))
    z1, _ = ln.forward(params, y)
    z2, _ = ln.forward(params, 1e5 * y)
    assert np.max(np.abs(z2 - 1e5 * z1)) <= 1e-9 * np.max(np.abs(z2))
