"""The heat-equation workload of Sec. 7.2 with B and Q the banded circulant
modified SOAR of Sec. 6.1 (WC4D_COV_MSOAR: built from (amp, L, maxval) and the
shift draws psi, applied through their 2 maxval + 1 taps, never dense),
against the FP64 oracle.

Tolerances (relative 2-norm): A v 1e-12 in FP64 mode (1e-11 with OZAKI / DF32
R-family products), P_I^{-1} v 1e-9, the small solve within 1e-8 of dense LU;
at the paper's full size (s = 50,000, N = 5, p = 12,500) A v against the
oracle's band-applied operator and a P_I + GMRES solve to 1e-6 with the
oracle's operator.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2105_06975_gb300 import workload as W

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2105_06975_gb300 import wc4d as L  # noqa: E402
from oracle import covariance as cov, problem as prb, saddle as sd  # noqa: E402

DEV = "cuda"


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def gpu(w, dr, model, opts, R=None):
    """The library problem: heat model bands, modified SOAR B and Q from their
    parameters and the workload's psi draws; R dense (given) or SOAR."""
    kw = dict(R=R) if R is not None else dict(soar_r=w.soar_r)
    return L.Problem(w.s, w.N, w.p, dr.obs_idx, opts, bands=model.bands, band_lo=model.lo, band_hi=model.hi,
                     msoar=(w.msoar_b, w.msoar_q, dr.extra["psi"]), **kw)


@pytest.mark.parametrize("precision", ["fp64", "df32", "ozaki"])
def test_heat_band_operators(precision):
    """s = 2000, N = 5, p = 500, channel-block R (passed dense)."""
    w = W.small(W.HEAT, s=2000, N=5, p=500)
    dr = W.draws(w, 1)
    prob, obs, rhs = prb.linear_case(w, dr)
    G = gpu(w, dr, prob.model, L.make_opts(precond="PI", k=3, precision=precision), R=prob.R)
    v = W.random_vector(prob.n, 3)
    tol_a = 1e-12 if precision == "fp64" else 1e-11
    assert rel(G.apply_saddle(to_dev(v)).cpu().numpy(), prob.A_apply(v)) < tol_a
    P = sd.Preconditioner(prob, sd.PrecondOptions(kind="PI", k=3))
    assert rel(G.apply_precond("PI", to_dev(v)).cpu().numpy(), P.apply(v)) < 1e-9
    G.close()


def test_heat_band_small_solve_matches_lu():
    w = W.small(W.HEAT, s=400, N=5, p=100)
    dr = W.draws(w, 2)
    prob, obs, rhs = prb.linear_case(w, dr)
    x_lu = sd.dense_solve(prob, rhs)
    G = gpu(w, dr, prob.model, L.make_opts(precond="PI", k=3, tol=1e-11, maxit=1000), R=prob.R)
    x, info = G.solve(to_dev(rhs))
    assert info.status == 0, L.wc4d_last_error()
    assert rel(x.cpu().numpy(), x_lu) < 1e-8
    G.close()


def test_heat_band_argument_checks():
    w = W.small(W.HEAT, s=400, N=5, p=100)
    dr = W.draws(w, 2)
    model = prb.linear_model(w)
    R = np.eye(w.p)
    for opts, needle in ((L.make_opts(precond="PD", k=2), "precond PI"),
                         (L.make_opts(precond="PI", k=2, covprod="fft"), "covprod DENSE")):
        with pytest.raises(L.WC4DError) as e:
            gpu(w, dr, model, opts, R=R)
        assert e.value.code == L.WC4D_ERR_ARG and needle in str(e.value)
    with pytest.raises(L.WC4DError) as e:
        L.Problem(w.s, w.N, w.p, dr.obs_idx, L.make_opts(precond="PI", k=2), bands=model.bands, band_lo=1,
                  band_hi=1, msoar=((0.4, 0.6, 300), w.msoar_q, dr.extra["psi"]), R=R)
    assert e.value.code == L.WC4D_ERR_ARG and "maxval" in str(e.value)


@pytest.mark.slow
def test_heat_full_size_band_solve():
    """Sec. 7.2 at its largest size: s = 50,000, N = 5, p = 12,500 observed
    points, R the chordal SOAR over them (sigma^2 = 0.5, 4-point length),
    right-hand side (0, z_r, 0).  A v within 1e-11 of the oracle's band-applied
    operator; P_I + GMRES with L_M(4) (OZAKI products) to 1e-6 with the
    oracle's operator."""
    w = W.HEAT_SOAR_R
    dr = W.draws(w, 0)
    prob = prb.heat_band_problem(w, dr)
    G = gpu(w, dr, prob.model, L.make_opts(precond="PI", k=4, precision="ozaki", tol=1e-6, maxit=1000))
    v = W.random_vector(prob.n, 5)
    assert rel(G.apply_saddle(to_dev(v)).cpu().numpy(), prob.A_apply(v)) < 1e-11
    rhs = prob.join(np.zeros((w.N + 1, w.s)), dr.z_r, np.zeros((w.N + 1, w.s)))
    x, info = G.solve(to_dev(rhs))
    assert info.status == 0, L.wc4d_last_error()
    r = rhs - prob.A_apply(x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(rhs) <= 1e-6
    print(f"heat full size: {info.iters} GMRES iterations, true relres {info.relres_true:.3e}, {info.ms:.0f} ms")
    G.close()
