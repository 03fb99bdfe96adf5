"""Parity of the CUDA library (through the C ABI) with the FP64 oracle.

Every case feeds both sides the same seeded inputs.  Tolerances (FP64 mode):
  * covariances, A v:                      1e-12 relative (2-norm)
  * P_I^{-1} v, P_D^{-1} v:                1e-9 relative (the library applies
    Dhat^{-1}, Rhat^{-1} through explicit inverse Cholesky factors; their error
    grows like kappa(L) eps, with kappa(L) = kappa(B)^{1/2} ~ 1e3 here)
  * solves:                                x within 1e-8 of dense LU when both
    are driven to 1e-12; true residual <= tol with the oracle's operator.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2105_06975_gb300 import workload as W

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2105_06975_gb300 import wc4d as L  # noqa: E402
from oracle import covariance as cov, krylov as kr, model as mdl, problem as prb, saddle as sd  # noqa: E402

DEV = "cuda"


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def case(s, N, p=None, obs="random", seed=0, base=W.TINY):
    w = W.small(base, s=s, N=N, p=p).with_(obs=obs)
    return w, W.draws(w, seed)


def popts(kind="PI", k=1, rhat="exact", shat="paper", dhat="exact", kappa=100.0):
    return sd.PrecondOptions(kind=kind, k=k, rhat=rhat, shat=shat, dhat=dhat, kappa_max=kappa)


def gpu_problem(w, dr, prob=None, precond="PI", k=1, rhat="exact", shat="paper", dhat="exact", kappa=100.0,
                krylov=None, tol=1e-6, maxit=1000, dense=False, banded=None):
    o = L.make_opts(precond=precond, k=k, rhat=rhat, kappa_max=kappa, shat=shat, dhat=dhat, krylov=krylov, tol=tol,
                    maxit=maxit)
    kw = {}
    if dense:
        kw.update(B=prob.B, Q=prob.Q, R=prob.R)
    if banded is not None:
        bands, lo, hi = banded
        kw.update(bands=bands, band_lo=lo, band_hi=hi)
        return L.Problem(w.s, w.N, w.p, dr.obs_idx, o, B=prob.B, Q=prob.Q, R=prob.R, **kw)
    return L.Problem.from_workload(w, dr, o, dense=dense, **kw)


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


# ------------------------------------------------------------ covariances
@pytest.mark.parametrize("s,N,p", [(100, 3, 50), (203, 2, 77)])
def test_soar_matrices(s, N, p):
    w, dr = case(s, N, p)
    prob = prb.linear_problem(w, dr)
    G = gpu_problem(w, dr)
    for which, ref in ((0, prob.B), (1, prob.Q), (2, prob.R)):
        got = G.matrix(which).cpu().numpy()
        assert rel(got, ref) < 1e-13, which
    G.close()


# ------------------------------------------------------------------- A v
@pytest.mark.parametrize("s,N,p,obs", [(100, 10, 50, "even"), (203, 5, 77, "random"), (64, 0, 64, "even"),
                                       (70, 3, 1, "random"), (130, 7, 130, "even")])
def test_apply_saddle(s, N, p, obs):
    w, dr = case(s, N, p, obs)
    prob = prb.linear_problem(w, dr)
    G = gpu_problem(w, dr)
    for seed in (1, 2):
        v = W.random_vector(prob.n, seed)
        got = G.apply_saddle(to_dev(v)).cpu().numpy()
        ref = prob.A_apply(v)
        assert rel(got, ref) < 1e-12
    G.close()


def banded_case(s=90, N=4, p=45, lo=5, hi=3, seed=3, scale=0.3):
    w, dr = case(s, N, p, "random", seed=seed)
    g = np.random.default_rng(seed)
    bands = scale * g.standard_normal((N, s, lo + hi + 1))
    B, Q, R = prb.covariances(w, dr.obs_idx)
    prob = sd.Problem(s, N, p, mdl.BandedModel(bands, lo, hi), np.asarray(dr.obs_idx), B, Q, R)
    return w, dr, prob, (bands, lo, hi)


def test_apply_saddle_banded_model():
    w, dr, prob, bd = banded_case()
    G = gpu_problem(w, dr, prob, banded=bd)
    v = W.random_vector(prob.n, 5)
    assert rel(G.apply_saddle(to_dev(v)).cpu().numpy(), prob.A_apply(v)) < 1e-12
    for kind in ("PI",):
        for k in (1, 2, 5):
            G2 = gpu_problem(w, dr, prob, precond=kind, k=k, banded=bd)
            P = sd.Preconditioner(prob, popts(kind, k))
            assert rel(G2.apply_precond(kind, to_dev(v)).cpu().numpy(), P.apply(v)) < 1e-9
            G2.close()
    G.close()


# ----------------------------------------------------------------- P^{-1} v
@pytest.mark.parametrize("kind", ["PD", "PI"])
@pytest.mark.parametrize("rhat", ["exact", "rr", "me", "diag"])
def test_apply_precond(kind, rhat):
    w, dr = case(120, 5, 61, "random")
    prob = prb.linear_problem(w, dr)
    v = W.random_vector(prob.n, 7)
    for k in (1, 2, 6):
        G = gpu_problem(w, dr, precond=kind, k=k, rhat=rhat)
        P = sd.Preconditioner(prob, popts(kind, k, rhat))
        got = G.apply_precond(kind, to_dev(v)).cpu().numpy()
        ref = P.apply(v)
        assert rel(got, ref) < 1e-9, (kind, rhat, k, rel(got, ref))
        if rhat in ("rr", "me"):
            Rh = G.matrix(3).cpu().numpy()
            assert rel(Rh, P.Rhat) < 1e-10
            lam = np.linalg.eigvalsh(prob.R)
            if rhat == "rr":
                assert G.rhat_param() == pytest.approx(cov.ridge_gamma(lam[0], lam[-1], 100.0), rel=1e-9)
            else:
                assert G.rhat_param() == pytest.approx(lam[-1] / 100.0, rel=1e-10)
        G.close()


def test_apply_precond_exact_schur_and_shifted_dhat():
    w, dr = case(40, 3, 20, "even")
    prob = prb.linear_problem(w, dr)
    v = W.random_vector(prob.n, 9)
    for kw in (dict(shat="exact"), dict(dhat="rr"), dict(shat="exact", rhat="rr")):
        G = gpu_problem(w, dr, precond="PD", k=2, **kw)
        P = sd.Preconditioner(prob, popts("PD", 2, kw.get("rhat", "exact"), kw.get("shat", "paper"),
                                          kw.get("dhat", "exact")))
        got = G.apply_precond("PD", to_dev(v)).cpu().numpy()
        assert rel(got, P.apply(v)) < 1e-8, kw
        G.close()


def test_synthesize_rhs_matches_oracle():
    """The device-built first-loop right-hand side (b, d, 0) equals the
    oracle's (truth, background and observations of the linear workload)."""
    for w, seed in ((W.TINY, 0), (W.small(W.SCALE, s=256, N=12, p=100), 3)):
        dr = W.draws(w, seed)
        prob, obs, rhs = prb.linear_case(w, dr)
        G = gpu_problem(w, dr)
        got = G.synthesize_rhs(dr).cpu().numpy()
        assert rel(got, rhs) < 1e-11
        assert np.all(got[:prob.s * (prob.N + 1)] == 0) and np.all(got[-prob.s * (prob.N + 1):] == 0)
        G.close()


# -------------------------------------------------------------------- solves
def test_tiny_config_mgw_minres_vs_lu():
    """Plain method on the tiny advection-diffusion workload: P_D with exact
    D, R and Schur complement; MINRES stops within a handful of iterations and
    matches dense LU."""
    w = W.TINY
    dr = W.draws(w, 0)
    prob, obs, rhs = prb.linear_case(w, dr)
    x_lu = sd.dense_solve(prob, rhs)
    G = gpu_problem(w, dr, precond="PD", shat="exact", krylov="minres", tol=1e-12, maxit=50)
    x, info = G.solve(to_dev(rhs))
    assert info.status == 0 and info.iters <= 5
    assert rel(x.cpu().numpy(), x_lu) < 1e-8
    G.close()


@pytest.mark.parametrize("kind,krylov,k,rhat", [("PD", "minres", 3, "exact"), ("PI", "gmres", 3, "rr"),
                                               ("PI", "gmres", 1, "exact"), ("PD", "gmres", 7, "me")])
def test_small_solves_match_lu_and_oracle_iterations(kind, krylov, k, rhat):
    w, dr = case(64, 6, 32, "random", seed=4)
    prob, obs, rhs = prb.linear_case(w, dr)
    x_lu = sd.dense_solve(prob, rhs)
    G = gpu_problem(w, dr, precond=kind, k=k, rhat=rhat, krylov=krylov, tol=1e-11, maxit=2000)
    x, info = G.solve(to_dev(rhs))
    assert info.status == 0, L.wc4d_last_error()
    # kappa(A) = 1.6e5 here; the oracle's own solves to 1e-11 land within
    # 1.3e-10 of LU, so the FP64 bound of 1e-8 holds with margin
    assert rel(x.cpu().numpy(), x_lu) < 1e-8
    G.close()
    # at the paper's tolerance the iteration counts agree with the oracle's
    G = gpu_problem(w, dr, precond=kind, k=k, rhat=rhat, krylov=krylov, tol=1e-6, maxit=1000)
    x, info = G.solve(to_dev(rhs))
    P = sd.Preconditioner(prob, popts(kind, k, rhat))
    from oracle import krylov as kr
    ref = (kr.minres if krylov == "minres" else kr.gmres)(prob.A_apply, P.apply, rhs, tol=1e-6)
    # the true-residual acceptance near 1e-6 may add a few iterations on
    # either side (rounding differs; the GPU re-checks on a tightened estimate)
    assert abs(info.iters - ref.iters) <= 2 + 0.05 * ref.iters, (info.iters, ref.iters)
    r = rhs - prob.A_apply(x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(rhs) <= 1e-6
    G.close()


def test_host_and_device_paths_agree_and_x0():
    w, dr = case(96, 4, 48, "random", seed=5)
    prob, obs, rhs = prb.linear_case(w, dr)
    G = gpu_problem(w, dr, precond="PI", k=5)
    xd, i1 = G.solve(to_dev(rhs))
    xh, i2 = G.solve(rhs.copy())
    assert np.array_equal(xd.cpu().numpy(), xh)
    assert i1.iters == i2.iters
    # restarting from the converged solution stops immediately
    x2, i3 = G.solve(to_dev(rhs), x=xd.clone(), use_x0=True)
    assert i3.iters <= 2 and i3.relres_true <= 1e-6
    G.close()


def test_banded_model_solve():
    w, dr, prob, bd = banded_case(s=80, N=5, p=40, lo=3, hi=2, seed=8, scale=0.12)
    rhs = W.random_vector(prob.n, 11)
    x_lu = sd.dense_solve(prob, rhs)
    G = gpu_problem(w, dr, prob, precond="PI", k=3, banded=bd, tol=1e-10, maxit=1000)
    x, info = G.solve(to_dev(rhs))
    assert info.status == 0
    # kappa(A) = 2.0e5; the oracle's solve to 1e-10 lands within 7e-12 of LU
    assert rel(x.cpu().numpy(), x_lu) < 1e-8
    G.close()


# ------------------------------------------------ double-float products
@pytest.mark.parametrize("kind", ["PD", "PI"])
def test_df32_operators_and_solve(kind):
    """DF32 mode (not in the paper): every covariance / factor product in
    double-float on the FP32 pipe.  A v within 1e-11 and P^{-1} v within 1e-9
    of the oracle (~48-bit products); the solve meets the true FP64 residual."""
    w, dr = case(203, 6, 77, "random", seed=2)
    prob, obs, rhs = prb.linear_case(w, dr)
    G = gpu_problem(w, dr, precond=kind, k=3)
    o = L.make_opts(precond=kind, k=3, precision="df32")
    D = L.Problem.from_workload(w, dr, o)
    v = W.random_vector(prob.n, 8)
    assert rel(D.apply_saddle(to_dev(v)).cpu().numpy(), prob.A_apply(v)) < 1e-11
    P = sd.Preconditioner(prob, popts(kind, 3))
    assert rel(D.apply_precond(kind, to_dev(v)).cpu().numpy(), P.apply(v)) < 1e-9
    x, info = D.solve(to_dev(rhs))
    _, i64 = G.solve(to_dev(rhs))
    assert info.status == 0
    assert abs(info.iters - i64.iters) <= 2 + 0.05 * i64.iters
    r = rhs - prob.A_apply(x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(rhs) <= 1e-6
    D.close()
    G.close()


def test_df32_gmres_delayed_reorthogonalisation():
    """DF32 GMRES runs the Arnoldi process with delayed reorthogonalisation
    (one dot pass and one update pass per step; Hessenberg column j-1 completed
    at step j).  The GMRES iterate after k steps is the unique minimiser over the
    k-dimensional Krylov space, so it must match the oracle's GMRES iterate at
    the same k; the converged solve matches LU; a nonzero x0 converges too."""
    w, dr = case(203, 6, 77, "random", seed=2)
    prob, obs, rhs = prb.linear_case(w, dr)
    P = sd.Preconditioner(prob, popts("PI", 3))
    for k in (1, 2, 7, 19):
        o = L.make_opts(precond="PI", k=3, precision="df32", tol=1e-14, maxit=k)
        D = L.Problem.from_workload(w, dr, o)
        x, info = D.solve(to_dev(rhs))
        ref = kr.gmres(prob.A_apply, P.apply, rhs, tol=1e-14, maxit=k)
        assert info.status == L.WC4D_ERR_MAXIT and info.iters == k, info.as_dict()
        assert rel(x.cpu().numpy(), ref.x) < 1e-7, k
        D.close()
    o = L.make_opts(precond="PI", k=3, precision="df32", tol=1e-10, maxit=300)
    D = L.Problem.from_workload(w, dr, o)
    x, info = D.solve(to_dev(rhs))
    ref = kr.gmres(prob.A_apply, P.apply, rhs, tol=1e-10, maxit=300)
    assert info.status == 0 and abs(info.iters - ref.iters) <= 1, (info.iters, ref.iters)
    x_lu = sd.dense_solve(prob, rhs)
    # kappa(A) = 1.3e7; the oracle's GMRES to 1e-10 lands within 1.2e-11 of LU
    assert rel(x.cpu().numpy(), x_lu) < 1e-8
    x0 = W.random_vector(prob.n, 5)
    x1, info1 = D.solve(to_dev(rhs), to_dev(x0), use_x0=True)
    assert info1.status == 0
    r = rhs - prob.A_apply(x1.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(rhs) <= 1e-10
    D.close()


@pytest.mark.parametrize("k", [1, 4])
def test_df32_gmres_fp32_preconditioner(k):
    """DF32_P32 mode (not in the paper): the preconditioner in FP32 inside the
    DF32 GMRES.  The stored preconditioned vectors make the iteration flexible,
    so the FP32 rounding of P^{-1} shows up as a few more iterations, not as a
    loss of accuracy: the true residual reaches 1e-10 and the solution matches
    LU like the DF32 mode's."""
    w, dr = case(203, 6, 77, "random", seed=2)
    prob, obs, rhs = prb.linear_case(w, dr)
    x_lu = sd.dense_solve(prob, rhs)
    res = {}
    for prec in ("df32", "df32p32"):
        o = L.make_opts(precond="PI", k=k, precision=prec, tol=1e-10, maxit=600)
        D = L.Problem.from_workload(w, dr, o)
        x, info = D.solve(to_dev(rhs))
        assert info.status == 0, (prec, info.as_dict())
        xg = x.cpu().numpy()
        r = rhs - prob.A_apply(xg)
        assert np.linalg.norm(r) / np.linalg.norm(rhs) <= 1e-10
        res[prec] = (info.iters, rel(xg, x_lu))
        D.close()
    assert res["df32p32"][0] <= 1.25 * res["df32"][0] + 3, res
    assert res["df32p32"][1] <= 10 * res["df32"][1] + 1e-9, res


# --------------------------------------------------------- mixed precision
@pytest.mark.parametrize("kind", ["PD", "PI"])
def test_fp32_operators(kind):
    """FP32 copies of A and P^{-1} (mixed mode) against the FP64 oracle at an
    FP32 bound: relative error <= 1e-5 (eps32 = 6e-8 times the growth of the
    factor products at these condition numbers)."""
    w, dr = case(96, 8, 48, "random", seed=6)
    prob = prb.linear_case(w, dr)[0]
    o = L.make_opts(precond=kind, k=4, precision="mixed", inner_iters=5, maxit=50)
    G = L.Problem.from_workload(w, dr, o)
    v = W.random_vector(prob.n, 2)
    v32 = torch.from_numpy(v.astype(np.float32)).cuda()
    vq = v32.double().cpu().numpy()           # the exact vector the FP32 path sees
    assert rel(G.apply_fp32("A", v32).double().cpu().numpy(), prob.A_apply(vq)) < 1e-5
    P = sd.Preconditioner(prob, popts(kind, 4))
    assert rel(G.apply_fp32(kind, v32).double().cpu().numpy(), P.apply(vq)) < 1e-5
    G.close()



@pytest.mark.parametrize("kind,k,rhat", [("PI", 4, "exact"), ("PI", 1, "rr"), ("PD", 3, "exact")])
def test_mixed_precision_fgmres(kind, k, rhat):
    """FP64 outer FGMRES around an FP32 inner GMRES(m) (not in the paper).

    At the paper's tolerance: converged, true FP64 residual <= 1e-6 recomputed
    with the oracle's operator, forward error vs dense LU <= 1e-4 (stated bound
    for this workload: kappa(B) = 4.6e5 lets a 1e-6 residual move x by up to
    ~1e-4; the FP64 mode lands within the same bound).  Driven to 1e-10 the
    mixed mode agrees with LU to 1e-7: the FP64 outer iteration recovers full
    accuracy from the FP32 inner solves (P_I)."""
    w, dr = case(96, 8, 48, "random", seed=6)
    prob, obs, rhs = prb.linear_case(w, dr)
    x_lu = sd.dense_solve(prob, rhs)
    G64 = gpu_problem(w, dr, precond=kind, k=k, rhat=rhat, tol=1e-6, maxit=1000)
    x64, i64 = G64.solve(to_dev(rhs))
    assert rel(x64.cpu().numpy(), x_lu) <= 1e-4
    G64.close()
    # P_D's inner D-hat^{-1} runs on FP32 factors of B (kappa 4.6e5): an FP32
    # inner solve with it stalls near 1e-3 on its own (CPU simulation with the
    # oracle), so only the paper's tolerance is asked of the nested P_D solve,
    # with 25 inner steps: with 15 the FP32 inner GMRES is too weak a
    # preconditioner and the outer FGMRES stagnates near 1e-5 (measured on the GPU)
    cases = ((1e-6, 1e-4), (1e-10, 1e-7)) if kind == "PI" else ((1e-6, 1e-4),)
    inner = 15 if kind == "PI" else 25
    for tol, bound in cases:
        o = L.make_opts(precond=kind, k=k, rhat=rhat, tol=tol, maxit=200, precision="mixed", inner_iters=inner)
        G = L.Problem.from_workload(w, dr, o)
        x, info = G.solve(to_dev(rhs))
        assert info.status == 0, L.wc4d_last_error()
        assert info.inner_iters == inner * info.iters
        # the nested solve needs far fewer FP64 operator applications
        assert info.iters <= i64.iters // 2, (info.iters, i64.iters)
        xm = x.cpu().numpy()
        r = rhs - prob.A_apply(xm)
        assert np.linalg.norm(r) / np.linalg.norm(rhs) <= tol
        assert rel(xm, x_lu) <= bound, (tol, rel(xm, x_lu))
        G.close()


# ------------------------------------------------ Lorenz-96 Gauss-Newton
def l96_gpu_gn(w, dr, obs, loops, tol, kind="PI", k=3, precision="fp64"):
    B, Q, R = prb.covariances(w, dr.obs_idx)
    lo, hi = mdl.band_width(w.steps_per_obs)
    o = L.make_opts(precond=kind, k=k, tol=tol, maxit=2000 if kind == "PI" else 5000, precision=precision)
    G = L.Problem(w.s, w.N, w.p, dr.obs_idx, o, banded=True, band_lo=lo, band_hi=hi, B=B, Q=Q, R=R)
    traj, infos, code = G.l96_gauss_newton(w.forcing, w.dt, w.steps_per_obs, loops, obs.xb, obs.y)
    G.close()
    return traj, infos, code


@pytest.mark.parametrize("loops", [1, 3])
def test_l96_gauss_newton_small(loops):
    """Incremental weak-constraint 4D-Var on Lorenz-96 (Sec. 2.1, 7.1): the
    GPU outer loop (RK4 forecasts, banded TLM by coloured probing, (b, d),
    inner saddle-point solve) follows the oracle's trajectory."""
    w = W.small(W.L96, s=80, N=4, p=40).with_(spinup_steps=300)
    dr = W.draws(w, 1)
    B, Q, R = prb.covariances(w, dr.obs_idx)
    obs = prb.l96_truth(w, dr, B, Q, R, dr.obs_idx)
    trajs, results, _ = prb.gauss_newton_l96(w, dr, popts("PI", 3), "gmres", tol=1e-11, maxit=3000, loops=loops,
                                             obs=obs)
    traj, infos, code = l96_gpu_gn(w, dr, obs, loops, 1e-11)
    assert code == 0 and all(i.status == 0 for i in infos)
    assert rel(traj, trajs[-1]) < 1e-8
    assert rel(traj, trajs[0]) > 1e-3          # the loop did move the trajectory


def test_l96_gauss_newton_small_ozaki():
    """The same outer loop with the covariance / factor products as exact BF16
    digit products on the tensor cores (OZAKI mode, not in the paper): the
    trajectory still follows the oracle's.  The inner solves run to 1e-8 (the
    batched path's tolerance): at 1e-11 the Pythagorean norm of the Arnoldi
    candidate reaches zero (reported as a breakdown) before the residual
    estimate does, the products carrying ~2^-44 of max|a| max|x| against
    FP64's 2^-53; the oracle's trajectory is taken at 1e-11."""
    w = W.small(W.L96, s=80, N=4, p=40).with_(spinup_steps=300)
    dr = W.draws(w, 1)
    B, Q, R = prb.covariances(w, dr.obs_idx)
    obs = prb.l96_truth(w, dr, B, Q, R, dr.obs_idx)
    trajs, results, _ = prb.gauss_newton_l96(w, dr, popts("PI", 3), "gmres", tol=1e-11, maxit=3000, loops=1,
                                             obs=obs)
    traj, infos, code = l96_gpu_gn(w, dr, obs, 1, 1e-8, precision="ozaki")
    assert code == 0 and all(i.status == 0 for i in infos)
    assert rel(traj, trajs[-1]) < 1e-6
    assert rel(traj, trajs[0]) > 1e-3


def l96_cost(w, obs, B, Q, R, obs_idx, traj):
    """Nonlinear weak-constraint cost (Eq. CostFn) of a trajectory."""
    e0 = traj[0] - obs.xb
    out = e0 @ np.linalg.solve(B, e0)
    for t in range(w.N + 1):
        e = obs.y[t] - traj[t, obs_idx]
        out += e @ np.linalg.solve(R, e)
    for t in range(1, w.N + 1):
        e = traj[t] - mdl.l96_forecast(traj[t - 1], w.dt, w.forcing, w.steps_per_obs)
        out += e @ np.linalg.solve(Q, e)
    return out


def test_l96_full_size_linearisation():
    """s=1000, N=50, 5 RK4 steps per window: about the background trajectory
    the GPU's right-hand side (b, d, 0), its A v with the rebuilt banded
    tangent-linear models and P_I^{-1} v agree with the oracle's."""
    w = W.L96
    dr = W.draws(w, 0)
    B, Q, R = prb.covariances(w, dr.obs_idx)
    obs = prb.l96_truth(w, dr, B, Q, R, dr.obs_idx)
    traj = prb.l96_background(w, obs.xb)
    bands, lo, hi = prb.l96_linearise(w, traj)
    prob = sd.Problem(w.s, w.N, w.p, mdl.BandedModel(bands, lo, hi), np.asarray(dr.obs_idx), B, Q, R)
    rhs = prb.l96_rhs(w, prob, obs, traj)
    o = L.make_opts(precond="PI", k=3, tol=1e-6, maxit=50)
    G = L.Problem(w.s, w.N, w.p, dr.obs_idx, o, banded=True, band_lo=lo, band_hi=hi, B=B, Q=Q, R=R)
    got = G.l96_linearize(w.forcing, w.dt, w.steps_per_obs, obs.xb, obs.y, traj)
    assert rel(got, rhs) < 1e-12
    v = W.random_vector(prob.n, 4)
    assert rel(G.apply_saddle(to_dev(v)).cpu().numpy(), prob.A_apply(v)) < 1e-11
    P = sd.Preconditioner(prob, popts("PI", 3))
    assert rel(G.apply_precond("PI", to_dev(v)).cpu().numpy(), P.apply(v)) < 1e-9
    G.close()


def l96_lin_cost(w, prob, rhs, dx, B, Q, R):
    """Linearised inner-loop cost J_lin(dx) = |L dx - b|^2_{D^-1} + |H dx - d|^2_{R^-1}
    (Sec. 2.1), blockwise with the oracle's L."""
    ns, npn = w.s * (w.N + 1), w.p * (w.N + 1)
    b = rhs[:ns].reshape(w.N + 1, w.s)
    d = rhs[ns:ns + npn].reshape(w.N + 1, w.p)
    e1 = mdl.L_apply(prob.model, dx) - b
    e2 = dx[:, prob.obs_idx] - d
    out = e1[0] @ np.linalg.solve(B, e1[0])
    out += sum(e1[t] @ np.linalg.solve(Q, e1[t]) for t in range(1, w.N + 1))
    out += sum(e2[t] @ np.linalg.solve(R, e2[t]) for t in range(w.N + 1))
    return float(out)


@pytest.mark.slow
def test_l96_gauss_newton_full_size():
    """One outer loop at s=1000, N=50 (5 RK4 steps of 0.025 per window) with
    P_I and Lhat = L (k = N+1, the strongest model information of Definition
    1).  Fifty windows of chaotic Lorenz-96 make the saddle-point system far
    harder than the paper's (Sec. 7.1 uses 15 windows of 1e-4): the true
    residual of the FP64 GMRES solve levels off near 1e-2 after about 1500
    iterations, and in a second outer loop it grows again before 2000
    iterations (the attainable accuracy of right-preconditioned GMRES shrinks
    with the norm of Lhat^{-1}, i.e. with the propagators over 50 windows).  So
    the full-size case runs one loop with the inner solve to 3e-2: it must meet
    that tolerance and at least halve the linearised cost J_lin (Sec. 2.1);
    measured on a GB300: 5.1e7 -> 7.4e6.  (The undamped step raises the nonlinear cost on this workload;
    the three-loop trajectory is checked against the oracle on the small case.)"""
    w = W.L96
    dr = W.draws(w, 0)
    B, Q, R = prb.covariances(w, dr.obs_idx)
    obs = prb.l96_truth(w, dr, B, Q, R, dr.obs_idx)
    traj0 = prb.l96_background(w, obs.xb)
    traj, infos, code = l96_gpu_gn(w, dr, obs, 1, 3e-2, k=w.N + 1)
    assert code == 0 and all(i.status == 0 for i in infos), [i.as_dict() for i in infos]
    bands, lo, hi = prb.l96_linearise(w, traj0)
    prob = sd.Problem(w.s, w.N, w.p, mdl.BandedModel(bands, lo, hi), np.asarray(dr.obs_idx), B, Q, R)
    rhs = prb.l96_rhs(w, prob, obs, traj0)
    dx = traj - traj0
    J0 = l96_lin_cost(w, prob, rhs, np.zeros_like(dx), B, Q, R)
    J1 = l96_lin_cost(w, prob, rhs, dx, B, Q, R)
    assert J1 < 0.5 * J0, (J0, J1)


# -------------------------------------------------------------------- errors
def test_argument_and_numerical_errors():
    w, dr = case(40, 3, 20, "even")
    prob = prb.linear_problem(w, dr)
    with pytest.raises(L.WC4DError) as e:
        gpu_problem(w, dr, k=0)
    assert e.value.code == L.WC4D_ERR_ARG
    bad = W.Draws(**{**dr.__dict__, "obs_idx": dr.obs_idx[::-1].copy()})
    with pytest.raises(L.WC4DError) as e:
        gpu_problem(w, bad)
    assert e.value.code == L.WC4D_ERR_ARG
    o = L.make_opts(precond="PD")
    Bneg = prob.B.copy()
    Bneg[0, 0] = -1.0
    with pytest.raises(L.WC4DError) as e:
        L.Problem(w.s, w.N, w.p, dr.obs_idx, o, stencil=w.stencil(), B=Bneg, Q=prob.Q, R=prob.R)
    assert e.value.code == L.WC4D_ERR_NOT_SPD
    Bnan = prob.B.copy()
    Bnan[3, 4] = np.nan
    with pytest.raises(L.WC4DError) as e:
        L.Problem(w.s, w.N, w.p, dr.obs_idx, o, stencil=w.stencil(), B=Bnan, Q=prob.Q, R=prob.R)
    assert e.value.code == L.WC4D_ERR_NONFINITE
    G = gpu_problem(w, dr, precond="PI")
    v = to_dev(W.random_vector(prob.n, 1))
    with pytest.raises(L.WC4DError) as e:
        G.apply_precond("PD", v)
    assert e.value.code == L.WC4D_ERR_ARG
    with pytest.raises(L.WC4DError):
        L.make_opts(precond="PI", krylov="minres") and gpu_problem(w, dr, precond="PI", krylov="minres")
    G.close()


def test_maxit_reports_status_and_last_iterate():
    w, dr = case(64, 6, 32, "random")
    prob, obs, rhs = prb.linear_case(w, dr)
    G = gpu_problem(w, dr, precond="PI", k=1, maxit=5)
    x, info = G.solve(to_dev(rhs))
    assert info.status == L.WC4D_ERR_MAXIT and info.iters == 5
    r = rhs - prob.A_apply(x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(rhs) == pytest.approx(info.relres_true, rel=1e-9)
    G.close()


# ------------------------------------------------------ full-size workload
@pytest.mark.slow
def test_scale_workload_operators_and_solve():
    """s=2048, N=64, p=1024 (n = 332,800), in the launch configuration the
    benchmark uses.

    * SOAR matrices built on the GPU agree with the oracle's entry by entry.
    * A v agrees to 1e-12 (with the oracle's own matrices passed in, and with
      the GPU-built ones).
    * P_I^{-1} v agrees to 1e-7.  kappa(R) = 2.6e9 and kappa(Q) = 5.6e9 here:
      two backward-stable FP64 Cholesky factorisations of the same R (the
      library's blocked one and LAPACK's) give R^{-1} v that differ by up to
      kappa(R) eps ~ 3e-7, and a 1e-16 relative perturbation of R's entries
      alone moves R^{-1} v by 1.5e-8 (measured with the oracle).  With the same
      factor, explicit inverse factors and triangular solves agree to 6e-14.
    * A solve meets the 1e-6 relative residual with the oracle's operator.
    """
    w = W.SCALE
    dr = W.draws(w, 0)
    prob, obs, rhs = prb.linear_case(w, dr)
    v = W.random_vector(prob.n, 3)
    P = sd.Preconditioner(prob, popts("PI", 4))
    Av, Pv = prob.A_apply(v), P.apply(v)
    Gd = gpu_problem(w, dr, prob, precond="PI", k=4, dense=True)
    assert rel(Gd.apply_saddle(to_dev(v)).cpu().numpy(), Av) < 1e-12
    assert rel(Gd.apply_precond("PI", to_dev(v)).cpu().numpy(), Pv) < 1e-7
    Gd.close()
    G = gpu_problem(w, dr, precond="PI", k=4)
    for which, ref in ((0, prob.B), (1, prob.Q), (2, prob.R)):
        assert rel(G.matrix(which).cpu().numpy(), ref) < 1e-13
    assert rel(G.apply_saddle(to_dev(v)).cpu().numpy(), Av) < 1e-12
    assert rel(G.apply_precond("PI", to_dev(v)).cpu().numpy(), Pv) < 1e-7
    x, info = G.solve(to_dev(rhs))
    assert info.status == 0
    r = rhs - prob.A_apply(x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(rhs) <= 1e-6
    G.close()


@pytest.mark.parametrize("kind,krylov,k,lhat", [("PD", "minres", 3, "lm"), ("PI", "gmres", 2, "lm"),
                                                ("PI", "gmres", 4, "i")])
def test_product_counts_follow_tables_4_5(kind, krylov, k, lhat):
    """wc4d_info's per-component product counts (Tables 4 and 5 convention: one
    count per time block a product touches).  The oracle's own operators,
    wrapped to count, give the products of one A apply and one P apply; the
    library's totals after 7 iterations must equal those per-apply counts times
    its own numbers of A and P applies, and those numbers follow the solver
    (7 preconditioner applies plus MINRES's initial one)."""
    w, dr = case(48, 5, 24, "random", seed=3)
    prob, obs, rhs = prb.linear_case(w, dr)
    o = sd.PrecondOptions(kind=kind, k=k, rhat="exact", lhat_identity=(lhat == "i"))
    P = sd.Preconditioner(prob, o)
    cnt = {"D": 0, "R": 0, "Dh": 0, "Rh": 0, "M": 0}

    def wrap(obj, name, key, per):
        f = getattr(obj, name)

        def g(*a):
            cnt[key] += per(*a)
            return f(*a)
        setattr(obj, name, g)
    T = prob.N + 1
    wrap(prob, "D_apply", "D", lambda *a: T)
    wrap(prob, "R_apply", "R", lambda *a: T)
    wrap(P, "Dhat_inv", "Dh", lambda *a: T)
    wrap(P, "Rhat_inv", "Rh", lambda *a: T)
    wrap(prob.model, "apply", "M", lambda *a: 1)
    wrap(prob.model, "apply_T", "M", lambda *a: 1)
    v = W.random_vector(prob.n, 2)
    prob.A_apply(v)
    perA = dict(cnt)
    for key in cnt:
        cnt[key] = 0
    P.apply(v)
    perP = dict(cnt)
    G = gpu_problem(w, dr, precond=kind, k=k, krylov=krylov, tol=1e-30, maxit=7)
    if lhat == "i":
        G.close()
        G = L.Problem.from_workload(w, dr, L.make_opts(precond=kind, k=k, krylov=krylov, tol=1e-30, maxit=7,
                                                       lhat="i"))
    x, info = G.solve(to_dev(rhs))
    assert info.status == L.WC4D_ERR_MAXIT and info.iters == 7
    nA, nP = info.n_apply_A, info.n_apply_P
    assert nP == 7 + (1 if krylov == "minres" else 0)
    assert info.n_R == nA * perA["R"] and perA["R"] == T
    assert info.n_D == nA * perA["D"] + nP * perP["D"]
    assert info.n_Dhat_inv == nP * perP["Dh"] and info.n_Rhat_inv == nP * perP["Rh"]
    assert info.n_M == nA * perA["M"] + nP * perP["M"]
    assert info.n_cov == info.n_R + info.n_D and info.n_trsm == info.n_Dhat_inv + info.n_Rhat_inv
    # the ratios Tables 4 and 5 print: D_i = 2 R_i per iteration, Dhat^-1 = R_i for P_D, none for P_I
    assert perP["D"] == perA["R"] and (perP["Dh"] == T if kind == "PD" else perP["Dh"] == 0)
    G.close()


@pytest.mark.parametrize("kind,precision,covprod", [("PI", "fp64", "dense"), ("PD", "fp64", "dense"),
                                                    ("PI", "ozaki", "dense"), ("PD", "df32", "fft"),
                                                    ("PI", "ozaki", "fft")])
def test_explicit_rhat_inverse(kind, precision, covprod):
    """rinv_explicit (not in the paper): Rhat^-1 = W^T W formed once at setup
    and applied as one product.  P^-1 v within 1e-9 of the oracle (as the
    factor pair), the solve within 1e-8 of LU in FP64 mode (1e-6 with the
    OZAKI products) in the factor pair's iteration count (+-(2 + 5 %))."""
    w, dr = case(128, 6, 48, "random", seed=9)
    prob, obs, rhs = prb.linear_case(w, dr)
    krylov = "minres" if kind == "PD" else "gmres"
    o = dict(precond=kind, k=3, krylov=krylov, precision=precision, covprod=covprod, tol=1e-11, maxit=2000)
    G = L.Problem.from_workload(w, dr, L.make_opts(rinv_explicit=True, **o))
    F = L.Problem.from_workload(w, dr, L.make_opts(**o))
    v = W.random_vector(prob.n, 12)
    P = sd.Preconditioner(prob, popts(kind, 3))
    assert rel(G.apply_precond(kind, to_dev(v)).cpu().numpy(), P.apply(v)) < 1e-9
    x_lu = sd.dense_solve(prob, rhs)
    x, info = G.solve(to_dev(rhs))
    _, info_f = F.solve(to_dev(rhs))
    # MINRES driven to 1e-11 moves its count by a few per cent under last-bit changes of P^-1 (the
    # oracle's own count does, too): the counts agree to 2 + 5 %
    assert info.status == 0 and abs(info.iters - info_f.iters) <= 2 + 0.05 * info_f.iters, (info.iters, info_f.iters)
    assert rel(x.cpu().numpy(), x_lu) < (1e-8 if precision == "fp64" else 1e-6)
    G.close()
    F.close()


@pytest.mark.slow
def test_explicit_rhat_inverse_scale_window():
    """At the scale window (kappa(R) = 2.6e9): P_I^{-1} v within 1e-7 of the
    oracle (the factor pair's bound, kappa(R) eps), and the OZAKI P_I + GMRES
    solve reaches 1e-6 with the oracle's operator in the factor pair's count
    (+-2, 5 %)."""
    w = W.SCALE
    dr = W.draws(w, 0)
    prob, obs, rhs = prb.linear_case(w, dr)
    its = {}
    for flag in (True, False):
        G = L.Problem.from_workload(w, dr, L.make_opts(precond="PI", k=4, precision="ozaki", tol=1e-6, maxit=1000,
                                                       rinv_explicit=flag))
        if flag:
            v = W.random_vector(prob.n, 13)
            P = sd.Preconditioner(prob, popts("PI", 4))
            assert rel(G.apply_precond("PI", to_dev(v)).cpu().numpy(), P.apply(v)) < 1e-7
        x, info = G.solve(to_dev(rhs))
        assert info.status == 0
        r = rhs - prob.A_apply(x.cpu().numpy())
        assert np.linalg.norm(r) / np.linalg.norm(rhs) <= 1e-6
        its[flag] = info.iters
        G.close()
    assert abs(its[True] - its[False]) <= 2 + 0.05 * its[False], its


@pytest.mark.parametrize("precision", ["df32", "ozaki"])
@pytest.mark.parametrize("tol", [1e-6, 1e-7])
def test_six_byte_basis(precision, tol):
    """basis_bytes = 6 (not in the paper): the delayed-CGS2 basis stored as
    FP32 high + BF16 low parts (about 32 significant bits).  The solve reaches
    tol with the oracle's operator, in the 8-byte basis's iteration count
    (+-(2 + 5 %)), and its solution agrees with the 8-byte basis's within
    100 tol (both are tol-accurate in the residual; kappa(A) is small here)."""
    w, dr = case(256, 8, 96, "random", seed=4)
    prob, obs, rhs = prb.linear_case(w, dr)
    o = dict(precond="PI", k=2, precision=precision, tol=tol, maxit=600)
    runs = {}
    for bb in (6, 8):
        G = L.Problem.from_workload(w, dr, L.make_opts(basis_bytes=bb, **o))
        x, info = G.solve(to_dev(rhs))
        assert info.status == 0, L.wc4d_last_error()
        xs = x.cpu().numpy()
        r = rhs - prob.A_apply(xs)
        assert np.linalg.norm(r) / np.linalg.norm(rhs) <= tol
        runs[bb] = (xs, info.iters)
        G.close()
    assert abs(runs[6][1] - runs[8][1]) <= 2 + 0.05 * runs[8][1], (runs[6][1], runs[8][1])
    assert rel(runs[6][0], runs[8][0]) < 100 * tol


@pytest.mark.slow
def test_six_byte_basis_scale_window():
    """At the scale window (kappa(B) about 1e11): the OZAKI P_I + GMRES solve
    with the explicit Rhat^-1 and the 6-byte basis reaches 1e-6 with the
    oracle's operator in the 8-byte basis's count (+-2, 5 %)."""
    w = W.SCALE
    dr = W.draws(w, 0)
    prob, obs, rhs = prb.linear_case(w, dr)
    its = {}
    for bb in (6, 8):
        G = L.Problem.from_workload(w, dr, L.make_opts(precond="PI", k=4, precision="ozaki", tol=1e-6, maxit=1000,
                                                       rinv_explicit=True, basis_bytes=bb))
        x, info = G.solve(to_dev(rhs))
        assert info.status == 0, L.wc4d_last_error()
        r = rhs - prob.A_apply(x.cpu().numpy())
        assert np.linalg.norm(r) / np.linalg.norm(rhs) <= 1e-6
        its[bb] = info.iters
        G.close()
    assert abs(its[6] - its[8]) <= 2 + 0.05 * its[8], its
