"""The heat-equation workload (Sec. 7.2) through the C ABI against the oracle.

The library has no heat-specific code: the Dirichlet model goes in as the
banded model kind (bands (r, 1-2r, r) inside, zero boundary rows and
columns), the modified SOAR B, Q and the channel-block R_i of Sec. 6.1 as
dense covariances.  Tolerances as in the other FP64 parity tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2105_06975_gb300 import workload as W

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2105_06975_gb300 import wc4d as L  # noqa: E402
from oracle import problem as prb, saddle as sd  # noqa: E402

DEV = "cuda"


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def heat_bands(s, N, r):
    """Sec. 7.2's M as the library's band input: row j, offsets -1, 0, +1."""
    bands = np.zeros((N, s, 3))
    for j in range(1, s - 1):
        bands[:, j, 0] = r if j - 1 >= 1 else 0.0
        bands[:, j, 1] = 1.0 - 2.0 * r
        bands[:, j, 2] = r if j + 1 <= s - 2 else 0.0
    return bands


def heat_case(s=96, N=3, p=24, seed=0):
    w = W.HEAT.with_(s=s, N=N, p=p, msoar_b=(0.4, 0.6, 8), msoar_q=(0.2, 0.5, 10), r_blocks=4,
                     r_msoar=(1.0, 0.5, 2))
    dr = W.draws(w, seed)
    prob, obs, rhs = prb.linear_case(w, dr)
    return w, dr, prob, rhs


def gpu(w, dr, prob, precond="PI", k=2, rhat="exact", tol=1e-10, precision="fp64"):
    o = L.make_opts(precond=precond, k=k, rhat=rhat, tol=tol, maxit=1000, precision=precision)
    return L.Problem(w.s, w.N, w.p, dr.obs_idx, o, B=prob.B, Q=prob.Q, R=prob.R,
                     bands=heat_bands(w.s, w.N, w.heat_r), band_lo=1, band_hi=1)


def test_heat_operators_match_oracle():
    w, dr, prob, rhs = heat_case()
    v = W.random_vector(prob.n, 3)
    G = gpu(w, dr, prob)
    assert rel(G.apply_saddle(torch.from_numpy(v).to(DEV)).cpu().numpy(), prob.A_apply(v)) < 1e-12
    G.close()
    for kind in ("PI", "PD"):
        for rhat in ("exact", "diag"):
            G = gpu(w, dr, prob, precond=kind, rhat=rhat)
            P = sd.Preconditioner(prob, sd.PrecondOptions(kind=kind, k=2, rhat=rhat))
            got = G.apply_precond(kind, torch.from_numpy(v).to(DEV)).cpu().numpy()
            assert rel(got, P.apply(v)) < 1e-9, (kind, rhat)
            G.close()


@pytest.mark.parametrize("precision", ["fp64", "df32"])
def test_heat_solve_matches_lu(precision):
    w, dr, prob, rhs = heat_case()
    x_lu = sd.dense_solve(prob, rhs)
    G = gpu(w, dr, prob, precond="PI", k=2, tol=1e-10, precision=precision)
    x, info = G.solve(torch.from_numpy(rhs).to(DEV))
    assert info.status == 0
    assert info.relres_true <= 1e-10
    assert rel(x.cpu().numpy(), x_lu) < 1e-8  # kappa(A) = 46: the oracle lands within 6e-11
    G.close()


# ------------------------------------------------ R_block (Alg. 3) and L_I
def gpu_opts(w, dr, prob, **kw):
    o = L.make_opts(maxit=1000, **kw)
    return L.Problem(w.s, w.N, w.p, dr.obs_idx, o, B=prob.B, Q=prob.Q, R=prob.R,
                     bands=heat_bands(w.s, w.N, w.heat_r), band_lo=1, band_hi=1)


def rblock_cases(R, pvec):
    """(tol, maxsize, numproc) cases with tol well away from every scaled norm
    (the two sides sum the norms in different orders)."""
    from oracle import covariance as cov
    nv = np.sort(cov.block_normvec(R, pvec))
    mids = [0.5 * (a + b) for a, b in zip(nv[:-1], nv[1:]) if b - a > 1e-6 * max(b, 1e-300)]
    cases = [(0.0, None, None), (np.inf, None, None), (0.0, 10, None), (np.inf, None, 3), (0.0, None, 6)]
    cases += [(m, None, None) for m in mids]
    return cases


def test_rblock_rhat_matches_oracle():
    from oracle import covariance as cov
    w, dr, prob, rhs = heat_case()
    pvec = W.block_sizes(w.p, w.r_blocks)
    for tol, maxsize, numproc in rblock_cases(prob.R, pvec):
        G = gpu_opts(w, dr, prob, rhat="block", rblock=(pvec, tol, maxsize, numproc))
        want = cov.r_block(prob.R, pvec, tol, maxsize, numproc)
        cuts, _ = cov.r_block_cuts(prob.R, pvec, tol, maxsize, numproc)
        assert np.array_equal(G.matrix(3).cpu().numpy(), want), (tol, maxsize, numproc)
        assert G.rhat_param() == len(cuts) + 1
        G.close()


@pytest.mark.parametrize("lhat", ["lm", "i"])
@pytest.mark.parametrize("kind", ["PI", "PD"])
def test_rblock_and_l_i_preconditioners_match_oracle(kind, lhat):
    w, dr, prob, rhs = heat_case()
    pvec = W.block_sizes(w.p, w.r_blocks)
    tol = rblock_cases(prob.R, pvec)[-1][0]
    v = W.random_vector(prob.n, 7)
    for k in (2, w.N + 1):
        G = gpu_opts(w, dr, prob, precond=kind, k=k, rhat="block", rblock=(pvec, tol, None, None), lhat=lhat)
        P = sd.Preconditioner(prob, sd.PrecondOptions(kind=kind, k=k, rhat="block", rblock=(pvec, tol, None, None),
                                                      lhat_identity=(lhat == "i")))
        got = G.apply_precond(kind, torch.from_numpy(v).to(DEV)).cpu().numpy()
        assert rel(got, P.apply(v)) < 1e-9, (k, lhat)
        G.close()


def test_rblock_l_i_solve_matches_lu():
    w, dr, prob, rhs = heat_case()
    pvec = W.block_sizes(w.p, w.r_blocks)
    tol = rblock_cases(prob.R, pvec)[-1][0]
    x_lu = sd.dense_solve(prob, rhs)
    G = gpu_opts(w, dr, prob, precond="PI", k=w.N + 1, rhat="block", rblock=(pvec, tol, None, None), lhat="i",
                 tol=1e-10)
    x, info = G.solve(torch.from_numpy(rhs).to(DEV))
    assert info.status == 0 and info.relres_true <= 1e-10
    assert rel(x.cpu().numpy(), x_lu) < 1e-8  # kappa(A) = 46: the oracle lands within 6e-11
    G.close()


def test_rblock_argument_errors():
    w, dr, prob, rhs = heat_case()
    for bad in [([5, 5], 0.1, None, None), ([0, 24], 0.1, None, None), ([12, 12], -1.0, None, None)]:
        with pytest.raises(L.WC4DError):
            gpu_opts(w, dr, prob, rhat="block", rblock=bad)
