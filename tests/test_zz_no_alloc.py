"""The allocation-free A v entry point agrees with the problem-handle one.

wc4d_apply_saddle_noalloc serves callers that cannot call cudaMalloc (a GPU
shared with a framework whose caching allocator holds the memory, or a loop
that cannot pay for allocation); it keeps its scratch in a fixed device array
inside the library.  Two calls in a row must both match wc4d_apply_saddle on
the same matrices, at the A v tolerance of the parity tests (1e-12), and the
FP64 oracle's blockwise A v at the same tolerance; an oversized
problem must be refused before any launch.  This file is collected last so
that a failure here does not hide the other GPU tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import model as mdl, problem as prb, saddle as sd  # noqa: E402
from paper_2105_06975_gb300 import wc4d as L, workload as W  # noqa: E402


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("s,N,p", [(2048, 64, 1024), (203, 5, 77), (64, 0, 64)])
def test_noalloc_matches_apply_saddle_twice(s, N, p):
    w = W.small(W.SCALE, s=s, N=N, p=p).with_(obs="random")
    dr = W.draws(w, 1)
    B, Q, R = prb.covariances(w, dr.obs_idx)
    opts = L.make_opts(precond="PI", k=1)
    G = L.Problem(w.s, w.N, w.p, dr.obs_idx, opts, stencil=w.stencil(), B=B, Q=Q, R=R)
    dev = torch.device("cuda")
    Bd, Qd, Rd = (torch.from_numpy(np.ascontiguousarray(M)).to(dev) for M in (B, Q, R))
    obs = torch.from_numpy(np.ascontiguousarray(dr.obs_idx, dtype=np.int32)).to(dev)
    stream = torch.cuda.current_stream().cuda_stream
    for seed in (3, 4):   # two calls in a row, different inputs
        v = torch.from_numpy(W.random_vector(w.n, seed)).to(dev)
        ref = G.apply_saddle(v)
        out = torch.full_like(v, float("nan"))
        L.wc4d_apply_saddle_noalloc(w.s, w.N, w.p, w.stencil(), obs.data_ptr(), Bd.data_ptr(), Qd.data_ptr(),
                                    Rd.data_ptr(), v.data_ptr(), out.data_ptr(), stream)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert rel(out, ref) < 1e-12
        prob = sd.Problem(s=w.s, N=w.N, p=w.p, model=mdl.StencilModel(w.s, w.N, w.stencil()),
                          obs_idx=np.asarray(dr.obs_idx), B=B, Q=Q, R=R)
        want = torch.from_numpy(prob.A_apply(v.cpu().numpy()))
        assert rel(out.cpu(), want) < 1e-12
    G.close()


def test_noalloc_rejects_oversized_problem():
    dev = torch.device("cuda")
    x = torch.zeros(8, dtype=torch.float64, device=dev)
    obs = torch.zeros(8, dtype=torch.int32, device=dev)
    with pytest.raises(L.WC4DError) as e:
        # 16384 grid points and 200 time levels need far more than 240 tiles
        L.wc4d_apply_saddle_noalloc(16384, 199, 8192, (0.7, 0.1, 0.2), obs.data_ptr(), x.data_ptr(), x.data_ptr(),
                                    x.data_ptr(), x.data_ptr(), x.data_ptr(), 0)
    assert e.value.code == L.WC4D_ERR_ARG
    assert "allocation-free" in str(e.value)
