"""Circulant covariance products by FFT (WC4D_COVPROD_FFT) against the FP64
oracle's dense products (Sec. 6.1: on the periodic uniform grid the SOAR B
and Q are circulant).

Tolerances (relative 2-norm):
  * A v, P_I^{-1} v in FP64 mode: 1e-12 / 1e-9, as the dense FP64 path (the
    transforms add ~log2(s) eps of the operator's scale);
  * Dhat^{-1} v1 of P_D: backward error ||Dhat y - v1|| <= 1e-12 (||Dhat|| ||y||
    + ||v1||) for y = Dhat^{-1} v1, the quantity both the FFT inverse and the
    oracle's Cholesky solve
    fix (their forward difference is bounded by kappa(B) eps, 1e-5 at the
    scale window, so it is compared at kappa-scaled tolerance);
  * solves: x within 1e-8 of dense LU (FP64 mode) on a small window; at the
    scale window the true residual with the oracle's operator <= 1e-6, in the
    iteration count of the dense-product solve (+-2, 5 %).
Shapes: s = 64 (Q = 8, one thread per 8-point DFT), 256, 2048; N = 0 (B only),
1 and odd N (an unpaired last column), 64.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2105_06975_gb300 import workload as W

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2105_06975_gb300 import wc4d as L  # noqa: E402
from oracle import krylov as kr, problem as prb, saddle as sd  # noqa: E402

DEV = "cuda"


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def case(s, N, p, seed=0, base=W.TINY):
    w = W.small(base, s=s, N=N, p=p).with_(obs="random")
    return w, W.draws(w, seed)


@pytest.mark.parametrize("s,N,p", [(64, 0, 32), (64, 1, 20), (256, 7, 100), (2048, 64, 1024), (512, 3, 512)])
@pytest.mark.parametrize("precision", ["fp64", "ozaki"])
def test_fft_apply_saddle_and_PI(s, N, p, precision):
    w, dr = case(s, N, p, seed=1)
    prob, obs, rhs = prb.linear_case(w, dr)
    G = L.Problem.from_workload(w, dr, L.make_opts(precond="PI", k=min(3, N + 1), precision=precision,
                                                   covprod="fft"))
    v = W.random_vector(prob.n, 4)
    tol_a = 1e-12 if precision == "fp64" else 1e-11
    assert rel(G.apply_saddle(to_dev(v)).cpu().numpy(), prob.A_apply(v)) < tol_a
    P = sd.Preconditioner(prob, sd.PrecondOptions(kind="PI", k=min(3, N + 1)))
    tol_p = 1e-9 if s <= 512 else 1e-7   # kappa(R) eps at the scale window, as the dense path
    assert rel(G.apply_precond("PI", to_dev(v)).cpu().numpy(), P.apply(v)) < tol_p
    G.close()


@pytest.mark.parametrize("dhat", ["exact", "rr"])
def test_fft_PD_blocks(dhat):
    """P_D^{-1} v with circulant Dhat^{-1}: the first block solves Dhat y = v1
    to a backward error of 1e-12; the third block (Lhat^{-1} D Lhat^{-T} v3,
    forward products only) and the second (Rhat^{-1}) match the oracle."""
    w, dr = case(256, 7, 100, seed=2)
    prob, obs, rhs = prb.linear_case(w, dr)
    G = L.Problem.from_workload(w, dr, L.make_opts(precond="PD", k=3, dhat=dhat, covprod="fft"))
    v = W.random_vector(prob.n, 6)
    out = G.apply_precond("PD", to_dev(v)).cpu().numpy()
    P = sd.Preconditioner(prob, sd.PrecondOptions(kind="PD", k=3, dhat=dhat))
    ref = P.apply(v)
    o1, o2, o3 = prob.split(out)
    r1, r2, r3 = prob.split(ref)
    v1 = prob.split(v)[0]
    delta = 0.01 if dhat == "rr" else 0.0
    Dh = prob.D_apply(o1) + delta * o1
    nD = max(np.linalg.norm(prob.B, 2), np.linalg.norm(prob.Q, 2)) + delta
    assert np.linalg.norm(Dh - v1) <= 1e-12 * (nD * np.linalg.norm(o1) + np.linalg.norm(v1))
    kB = np.linalg.cond(prob.B + delta * np.eye(prob.s))
    assert rel(o1, r1) < max(1e-12, 50 * kB * 2.2e-16)
    assert rel(o2, r2) < 1e-9 and rel(o3, r3) < 1e-11
    G.close()


@pytest.mark.parametrize("kind,krylov", [("PD", "minres"), ("PI", "gmres")])
def test_fft_small_solves_match_lu(kind, krylov):
    w, dr = case(64, 6, 32, seed=4)
    prob, obs, rhs = prb.linear_case(w, dr)
    x_lu = sd.dense_solve(prob, rhs)
    G = L.Problem.from_workload(w, dr, L.make_opts(precond=kind, k=3, krylov=krylov, tol=1e-11, maxit=2000,
                                                   covprod="fft"))
    x, info = G.solve(to_dev(rhs))
    assert info.status == 0, L.wc4d_last_error()
    assert rel(x.cpu().numpy(), x_lu) < 1e-8
    G.close()


@pytest.mark.slow
@pytest.mark.parametrize("kind,precision", [("PI", "ozaki"), ("PD", "ozaki"), ("PD", "fp64")])
def test_fft_scale_window_solve(kind, precision):
    """The scale window (s=2048, N=64, p=1024) with circulant products: the
    solve meets 1e-6 with the oracle's operator and takes the iteration count
    of the dense-product solve of the same mode (+-2, 5 %)."""
    w = W.SCALE
    dr = W.draws(w, 0)
    prob, obs, rhs = prb.linear_case(w, dr)
    krylov = "minres" if kind == "PD" else "gmres"
    maxit = 3000 if kind == "PD" else 1000
    its = {}
    for cp in ("fft", "dense"):
        G = L.Problem.from_workload(w, dr, L.make_opts(precond=kind, k=4, krylov=krylov, tol=1e-6, maxit=maxit,
                                                       precision=precision, covprod=cp))
        x, info = G.solve(to_dev(rhs))
        assert info.status == 0, (cp, L.wc4d_last_error())
        r = rhs - prob.A_apply(x.cpu().numpy())
        assert np.linalg.norm(r) / np.linalg.norm(rhs) <= 1e-6, cp
        its[cp] = info.iters
        G.close()
    assert abs(its["fft"] - its["dense"]) <= 2 + 0.05 * its["dense"], its


def test_fft_dense_covariances_and_errors():
    """Caller-given dense B, Q: accepted when circulant (then identical to the
    library-built SOAR case), refused with ARG when not; sizes the FFT does not
    handle and the FP32 modes are refused with ARG before any device work."""
    w, dr = case(128, 3, 40, seed=5)
    prob, obs, rhs = prb.linear_case(w, dr)
    o = L.make_opts(precond="PI", k=2, covprod="fft")
    G = L.Problem.from_workload(w, dr, o, dense=True, B=prob.B, Q=prob.Q, R=prob.R)
    v = W.random_vector(prob.n, 3)
    assert rel(G.apply_saddle(to_dev(v)).cpu().numpy(), prob.A_apply(v)) < 1e-12
    G.close()
    Bn = prob.B.copy()
    Bn[5, 9] += 1e-3
    Bn[9, 5] += 1e-3
    with pytest.raises(L.WC4DError) as e:
        L.Problem.from_workload(w, dr, o, dense=True, B=Bn, Q=prob.Q, R=prob.R)
    assert e.value.code == L.WC4D_ERR_ARG and "not circulant" in str(e.value)
    w2, dr2 = case(96, 3, 40, seed=5)
    with pytest.raises(L.WC4DError) as e:
        L.Problem.from_workload(w2, dr2, o)
    assert e.value.code == L.WC4D_ERR_ARG and "power of two" in str(e.value)
    with pytest.raises(L.WC4DError) as e:
        L.Problem.from_workload(w, dr, L.make_opts(precond="PI", k=2, precision="mixed", covprod="fft"))
    assert e.value.code == L.WC4D_ERR_ARG


def test_fft_product_counts_and_launches():
    """The FFT path keeps the Tables 4-5 product counts of the dense path (one
    D_i per time block per product, whatever the kernel)."""
    w, dr = case(256, 7, 100, seed=7)
    prob, obs, rhs = prb.linear_case(w, dr)
    infos = {}
    for cp in ("fft", "dense"):
        G = L.Problem.from_workload(w, dr, L.make_opts(precond="PD", k=3, krylov="minres", tol=1e-30, maxit=9,
                                                       covprod=cp))
        _, infos[cp] = G.solve(to_dev(rhs))
        G.close()
    for f in ("n_apply_A", "n_apply_P", "n_R", "n_D", "n_Dhat_inv", "n_Rhat_inv", "n_M"):
        assert getattr(infos["fft"], f) == getattr(infos["dense"], f), f
