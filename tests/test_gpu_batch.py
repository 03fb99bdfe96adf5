"""Batched solve of independent windows (wc4d_solve_batch; not in the paper).

Every window of a mixed batch (advection-diffusion and Lorenz-96 models,
uneven s, N, p, FP64 and DF32 modes, P_D + MINRES and P_I + GMRES) must come
out of the batch bit for bit equal to its own wc4d_solve: the batch runs the
same deterministic kernels on a worker stream.  Each solution is checked
against the oracle's operator (true residual) as in the single-window tests."""
import os
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import model as mdl, problem as prb, saddle as sd  # noqa: E402
from paper_2105_06975_gb300 import wc4d as L, workload as W  # noqa: E402

DEV = torch.device("cuda", 0)


def linear_window(s, N, p, seed, precond, precision):
    w = W.small(W.TINY, s=s, N=N, p=p).with_(obs="random")
    dr = W.draws(w, seed)
    prob, obs, rhs = prb.linear_case(w, dr)
    o = L.make_opts(precond=precond, k=3, precision=precision, tol=1e-8, maxit=600)
    return prob, rhs, L.Problem.from_workload(w, dr, o)


def l96_window(s, N, seed, precision):
    w = W.small(W.L96, s=s, N=N, p=s // 2).with_(steps_per_obs=2, spinup_steps=300)
    dr = W.draws(w, seed)
    B, Q, R = prb.covariances(w, dr.obs_idx)
    obs = prb.l96_truth(w, dr, B, Q, R, dr.obs_idx)
    traj = prb.l96_background(w, obs.xb)
    bands, lo, hi = prb.l96_linearise(w, traj)
    prob = sd.Problem(w.s, w.N, w.p, mdl.BandedModel(bands, lo, hi), np.asarray(dr.obs_idx), B, Q, R)
    rhs = prb.l96_rhs(w, prob, obs, traj)
    o = L.make_opts(precond="PI", k=N + 1, precision=precision, tol=1e-8, maxit=1500)
    G = L.Problem(w.s, w.N, w.p, dr.obs_idx, o, bands=bands, band_lo=lo, band_hi=hi, B=B, Q=Q, R=R)
    return prob, rhs, G


def batch():
    specs = [linear_window(96, 4, 48, 11, "PI", "df32"), linear_window(160, 2, 40, 12, "PD", "fp64"),
             linear_window(128, 7, 64, 13, "PI", "fp64"), linear_window(64, 3, 16, 14, "PI", "df32"),
             l96_window(80, 3, 15, "df32"), linear_window(200, 5, 100, 16, "PD", "fp64"),
             l96_window(96, 2, 17, "fp64"), linear_window(72, 9, 36, 18, "PI", "df32"),
             linear_window(144, 6, 70, 19, "PI", "ozaki"), l96_window(80, 4, 20, "ozaki")]
    return specs


@pytest.mark.parametrize("workers", [0, 3])
def test_batch_equals_individual_solves(workers):
    specs = batch()
    rhs_dev = [torch.from_numpy(r).to(DEV) for _, r, _ in specs]
    single = []
    for (prob, rhs, G), r in zip(specs, rhs_dev):
        x, info = G.solve(r)
        assert info.status == 0, info.as_dict()
        single.append(x.clone())
    xs, infos, code = L.solve_batch([G for _, _, G in specs], rhs_dev, workers=workers)
    assert code == 0
    for i, ((prob, rhs, G), x, x1, info) in enumerate(zip(specs, xs, single, infos)):
        assert info.status == 0, (i, info.as_dict())
        assert torch.equal(x, x1), i
        xn = x.cpu().numpy()
        assert np.linalg.norm(rhs - prob.A_apply(xn)) / np.linalg.norm(rhs) <= 1e-8 * 1.01, i
    # host buffers through the same call
    xs_h, infos_h, code_h = L.solve_batch([G for _, _, G in specs], [r for _, r, _ in specs], workers=workers)
    assert code_h == 0
    for x, x1 in zip(xs_h, single):
        assert np.array_equal(x, x1.cpu().numpy())
    for _, _, G in specs:
        G.close()


def test_batch_reports_failing_window_and_rejects_duplicates():
    a = linear_window(96, 4, 48, 21, "PI", "df32")
    prob, rhs, _ = a
    w = W.small(W.TINY, s=96, N=4, p=48).with_(obs="random")
    dr = W.draws(w, 21)
    tight = L.Problem.from_workload(w, dr, L.make_opts(precond="PI", k=1, tol=1e-12, maxit=3))
    r = [torch.from_numpy(rhs).to(DEV)] * 2
    xs, infos, code = L.solve_batch([a[2], tight], r)
    assert code == L.WC4D_ERR_MAXIT
    assert infos[0].status == 0 and infos[1].status == L.WC4D_ERR_MAXIT and infos[1].iters == 3
    assert "window 1" in L.wc4d_last_error()
    with pytest.raises(L.WC4DError):
        L.solve_batch([a[2], a[2]], r)
    a[2].close()
    tight.close()
