"""Per-time observation sets H_i and covariances R_i (Sec. 2.1: H and R are
block diagonal over the time levels) through the C ABI, against the FP64
oracle's PerTimeProblem / PerTimePreconditioner on the same seeded inputs.

Tolerances (relative 2-norm), as the shared-set parity tests:
  * A v 1e-12 (FP64 products in every mode for the R_i blocks; DF32 / OZAKI
    D products 1e-11);
  * P_I^{-1} v, P_D^{-1} v 1e-9;
  * identical sets at every time reproduce the shared-set problem to 1e-13;
  * solves: x within 1e-8 of dense LU (FP64 mode); the scale window's solve
    meets 1e-6 with the oracle's operator.
Cases cover sets of different sizes p_i per time (including p_i = 1 and
p_i = s), Rhat = R, R_diag, R_RR and R_ME per block, and the circulant FFT D
products together with per-time R_i.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2105_06975_gb300 import workload as W

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2105_06975_gb300 import wc4d as L  # noqa: E402
from oracle import covariance as cov, krylov as kr, problem as prb, saddle as sd  # noqa: E402

DEV = "cuda"


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def pertime_case(s, N, p, seed=0, sizes=None):
    """The workload's per-time draws, or (sizes given) sets of those sizes drawn
    from the same generator after the workload's draws."""
    w = W.small(W.TINY, s=s, N=N, p=p).with_(obs="random", obs_per_time=True)
    dr = W.draws(w, seed)
    if sizes is not None:
        g = np.random.default_rng(1000 + seed)
        dr.extra["obs_list"] = [np.sort(g.choice(s, size=k, replace=False)).astype(np.int32) for k in sizes]
    prob = prb.per_time_problem(w, dr)
    return w, dr, prob


def gpu(w, dr, prob, **kw):
    return L.Problem.from_workload(w, dr, L.make_opts(**kw), obs_list=prob.obs_list)


@pytest.mark.parametrize("sizes", [None, [1, 7, 64, 30, 33, 2]])
def test_pertime_apply_saddle(sizes):
    w, dr, prob = pertime_case(64, 5, 20, seed=1, sizes=sizes)
    G = gpu(w, dr, prob, precond="PI", k=2)
    v = W.random_vector(prob.n, 4)
    assert G.n == prob.n
    assert rel(G.apply_saddle(to_dev(v)).cpu().numpy(), prob.A_apply(v)) < 1e-12
    G.close()


@pytest.mark.parametrize("kind,rhat", [("PI", "exact"), ("PI", "diag"), ("PD", "rr"), ("PD", "me"),
                                       ("PI", "me")])
def test_pertime_preconditioners(kind, rhat):
    w, dr, prob = pertime_case(96, 6, 40, seed=2, sizes=[40, 12, 96, 5, 40, 60, 1])
    G = gpu(w, dr, prob, precond=kind, k=3, rhat=rhat, kappa_max=50.0)
    P = sd.PerTimePreconditioner(prob, sd.PrecondOptions(kind=kind, k=3, rhat=rhat, kappa_max=50.0))
    v = W.random_vector(prob.n, 5)
    assert rel(G.apply_precond(kind, to_dev(v)).cpu().numpy(), P.apply(v)) < 1e-9
    # Rhat_i blocks as the oracle builds them, one after another
    got = torch.empty(sum(len(o) ** 2 for o in prob.obs_list), dtype=torch.float64, device=DEV)
    L.load().wc4d_get_matrix(G.h, 3, L.ctypes.c_void_p(got.data_ptr()))
    want = np.concatenate([Rh.ravel(order="F") for Rh in P.Rhat_list])
    assert rel(got.cpu().numpy(), want) < 1e-10
    G.close()


def test_identical_sets_reduce_to_the_shared_problem():
    w = W.small(W.TINY, s=80, N=4, p=30).with_(obs="random")
    dr = W.draws(w, 3)
    shared = L.Problem.from_workload(w, dr, L.make_opts(precond="PD", k=2))
    per = L.Problem.from_workload(w, dr, L.make_opts(precond="PD", k=2), obs_list=[dr.obs_idx] * (w.N + 1))
    v = to_dev(W.random_vector(w.n, 6))
    assert rel(per.apply_saddle(v).cpu().numpy(), shared.apply_saddle(v).cpu().numpy()) < 1e-13
    for kind in ("PD", "PI"):
        assert rel(per.apply_precond(kind, v).cpu().numpy(), shared.apply_precond(kind, v).cpu().numpy()) < 1e-12
    shared.close()
    per.close()


@pytest.mark.parametrize("kind,krylov", [("PD", "minres"), ("PI", "gmres")])
def test_pertime_solve_matches_lu(kind, krylov):
    w, dr, prob = pertime_case(64, 6, 24, seed=4)
    _, _, rhs = prb.per_time_case(w, dr)
    x_lu = sd.dense_solve(prob, rhs)
    G = gpu(w, dr, prob, precond=kind, k=3, krylov=krylov, tol=1e-11, maxit=2000)
    x, info = G.solve(to_dev(rhs))
    assert info.status == 0, L.wc4d_last_error()
    assert rel(x.cpu().numpy(), x_lu) < 1e-8
    G.close()


@pytest.mark.parametrize("precision,covprod", [("df32", "dense"), ("ozaki", "dense"), ("ozaki", "fft"),
                                               ("fp64", "fft")])
def test_pertime_reduced_modes_and_fft(precision, covprod):
    w, dr, prob = pertime_case(128, 9, 50, seed=5)
    _, _, rhs = prb.per_time_case(w, dr)
    G = gpu(w, dr, prob, precond="PI", k=3, precision=precision, covprod=covprod, tol=1e-10, maxit=1000)
    v = W.random_vector(prob.n, 7)
    tol_a = 1e-12 if precision == "fp64" else 1e-11
    assert rel(G.apply_saddle(to_dev(v)).cpu().numpy(), prob.A_apply(v)) < tol_a
    P = sd.PerTimePreconditioner(prob, sd.PrecondOptions(kind="PI", k=3))
    assert rel(G.apply_precond("PI", to_dev(v)).cpu().numpy(), P.apply(v)) < 1e-9
    x, info = G.solve(to_dev(rhs))
    assert info.status == 0
    r = rhs - prob.A_apply(x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(rhs) <= 1e-10
    G.close()


@pytest.mark.slow
def test_pertime_scale_window():
    """s=2048, N=64, p_i=1024 per time (65 distinct sets and R_i blocks,
    545 MB per R-family operator): A v against the oracle and a P_I + GMRES
    solve (OZAKI D products) to 1e-6 with the oracle's operator."""
    w = W.SCALE.with_(obs_per_time=True)
    dr = W.draws(w, 0)
    prob, obs, rhs = prb.per_time_case(w, dr)
    G = L.Problem.from_workload(w, dr, L.make_opts(precond="PI", k=4, precision="ozaki", tol=1e-6, maxit=1000))
    v = W.random_vector(prob.n, 8)
    assert rel(G.apply_saddle(to_dev(v)).cpu().numpy(), prob.A_apply(v)) < 1e-11
    x, info = G.solve(to_dev(rhs))
    assert info.status == 0, L.wc4d_last_error()
    r = rhs - prob.A_apply(x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(rhs) <= 1e-6
    G.close()


def test_pertime_argument_checks():
    w, dr, prob = pertime_case(64, 3, 20, seed=6)
    with pytest.raises(L.WC4DError) as e:
        gpu(w, dr, prob, precond="PI", k=2, rhat="block", rblock=([10, 10], 0.1, None, None))
    assert e.value.code == L.WC4D_ERR_ARG
    bad = [o.copy() for o in prob.obs_list]
    bad[2] = bad[2][::-1].copy()
    with pytest.raises(L.WC4DError) as e:
        L.Problem.from_workload(w, dr, L.make_opts(precond="PI", k=2), obs_list=bad)
    assert e.value.code == L.WC4D_ERR_ARG and "strictly increasing" in str(e.value)
    G = gpu(w, dr, prob, precond="PI", k=2)
    with pytest.raises(L.WC4DError):
        G.synthesize_rhs(dr)
    G.close()
