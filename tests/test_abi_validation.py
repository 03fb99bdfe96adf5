"""wc4d_setup_problem's argument checks (host logic, no GPU): every invalid
descriptor or option is refused with WC4D_ERR_ARG and a message naming the
rule, before any device work, and no handle is returned."""
import ctypes

import numpy as np
import pytest

from paper_2105_06975_gb300 import build as B
from paper_2105_06975_gb300 import wc4d as L


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


def base(s=16, N=2, p=8):
    d = L.ProblemDesc()
    d.s, d.N, d.p = s, N, p
    d.model_kind = L.WC4D_MODEL_STENCIL3
    d.stencil[:] = [0.7, 0.1, 0.2]
    obs = np.arange(0, 2 * p, 2, dtype=np.int32)[:p]
    d.obs_idx = obs.ctypes.data
    d.cov_kind = L.WC4D_COV_SOAR
    d.soar_b[:] = [1.0, 0.1]
    d.soar_q[:] = [0.05, 0.05]
    d.soar_r[:] = [0.1, 0.05]
    d.mem_kind = L.WC4D_MEM_HOST
    return d, obs


def refused(lib, d, o, needle):
    h = ctypes.c_void_p()
    rc = lib.wc4d_setup_problem(ctypes.byref(d), ctypes.byref(o), None, ctypes.byref(h))
    msg = lib.wc4d_last_error().decode()
    if h.value:
        lib.wc4d_destroy(h)
    assert rc == L.WC4D_ERR_ARG, (rc, msg)
    assert needle in msg, msg
    assert not h.value


DESC_CASES = [
    ({"s": 1, "p": 1}, "need s >= 2"),
    ({"p": 17}, "1 <= p <= s"),
    ({"N": -1}, "N >= 0"),
    ({"mem_kind": 5}, "bad mem_kind"),
    ({"obs_idx": None}, "obs_idx is null"),
    ({"model_kind": 7}, "bad model_kind"),
    ({"model_kind": L.WC4D_MODEL_BANDED, "band_lo": 10, "band_hi": 6}, "band offsets"),
    ({"cov_kind": 9}, "bad cov_kind"),
    ({"cov_kind": L.WC4D_COV_DENSE}, "dense covariances missing"),
]


@pytest.mark.parametrize("edits,needle", DESC_CASES)
def test_descriptor_checks(lib, edits, needle):
    d, obs = base()
    for k, v in edits.items():
        setattr(d, k, v)
    refused(lib, d, L.make_opts(), needle)


def test_soar_parameters_positive(lib):
    d, obs = base()
    d.soar_q[1] = 0.0
    refused(lib, d, L.make_opts(), "SOAR variances and lengths")


OPT_CASES = [
    ({"precond": 5}, "bad precond"),
    ({"k": 0}, "k must lie in [1, N+1]"),
    ({"k": 4}, "k must lie in [1, N+1]"),
    ({"rhat": 9}, "bad rhat"),
    ({"rhat": L.WC4D_RHAT_RR, "kappa_max": 1.0}, "kappa_max must exceed 1"),
    ({"lhat": 3}, "bad lhat"),
    ({"shat": 7}, "bad shat"),
    ({"shat": L.WC4D_SHAT_LEARNED}, "learned Schur block"),
    ({"dhat": 4}, "bad dhat"),
    ({"krylov": 9}, "bad krylov"),
    ({"krylov": L.WC4D_KRYLOV_MINRES}, "MINRES needs"),
    ({"tol": 0.0}, "need tol > 0"),
    ({"maxit": 0}, "1 <= maxit"),
    ({"maxit": 3000}, "maxit <= 2000"),
    ({"precision": 9}, "bad precision"),
    ({"precision": L.WC4D_PREC_MIXED}, "mixed-precision mode is FGMRES"),
    ({"krylov": L.WC4D_KRYLOV_FGMRES}, "mixed-precision mode is FGMRES"),
    ({"precision": L.WC4D_PREC_MIXED, "krylov": L.WC4D_KRYLOV_FGMRES, "inner_iters": 0}, "inner_iters"),
    ({"precision": L.WC4D_PREC_DF32_P32, "precond": L.WC4D_PRECOND_PD, "krylov": L.WC4D_KRYLOV_MINRES},
     "FP32-preconditioner mode"),
]


@pytest.mark.parametrize("edits,needle", OPT_CASES)
def test_option_checks(lib, edits, needle):
    d, obs = base()
    o = L.make_opts()
    for k, v in edits.items():
        setattr(o, k, v)
    refused(lib, d, o, needle)


@pytest.mark.parametrize("s,edits,needle", [
    (16, {}, "power of two in [64, 8192]"),                 # base s = 16: below the FFT's smallest size
    (96, {}, "power of two in [64, 8192]"),
    (64, {"precision": L.WC4D_PREC_MIXED, "krylov": L.WC4D_KRYLOV_FGMRES}, "covprod FFT runs with precision"),
    (64, {"precision": L.WC4D_PREC_DF32_P32}, "covprod FFT runs with precision"),
    (64, {"precond": L.WC4D_PRECOND_PD, "krylov": L.WC4D_KRYLOV_MINRES, "shat": L.WC4D_SHAT_EXACT},
     "exact Schur complement"),
    (64, {"covprod": 5}, "bad covprod"),
])
def test_fft_covprod_checks(lib, s, edits, needle):
    d, obs = base(s=s, N=2, p=8)
    o = L.make_opts(covprod="fft")
    for k, v in edits.items():
        setattr(o, k, v)
    refused(lib, d, o, needle)


@pytest.mark.parametrize("counts,opt_edits,needle", [
    ([4, 4, 3], {}, "must sum to p"),                       # p = 12 in the descriptor
    ([4, 0, 8], {}, "must lie in [1, s]"),
    ([4, 4, 17], {}, "must lie in [1, s]"),
    ([4, 4, 4], {"rhat": L.WC4D_RHAT_BLOCK}, "rhat EXACT, DIAG, RR or ME"),
    ([4, 4, 4], {"precond": L.WC4D_PRECOND_PD, "krylov": L.WC4D_KRYLOV_MINRES, "shat": L.WC4D_SHAT_EXACT},
     "shat PAPER"),
    ([4, 4, 4], {"precision": L.WC4D_PREC_MIXED, "krylov": L.WC4D_KRYLOV_FGMRES}, "precision FP64, DF32 or OZAKI"),
])
def test_per_time_checks(lib, counts, opt_edits, needle):
    d, obs = base(s=16, N=2, p=12)
    pt = np.array(counts, dtype=np.int32)
    d.p_t = pt.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    allobs = np.concatenate([np.arange(max(c, 1), dtype=np.int32) for c in counts])
    d.obs_idx = allobs.ctypes.data
    o = L.make_opts()
    for k, v in opt_edits.items():
        setattr(o, k, v)
    refused(lib, d, o, needle)


def test_exact_schur_size_limit(lib):
    d, obs = base(s=4096, N=2, p=8)
    refused(lib, d, L.make_opts(precond="PD", shat="exact"), "exact Schur complement limited")


@pytest.mark.parametrize("rblock,needle", [
    (([4, 3], 0.1, None, None), "sum to p"),
    (([8, 0], 0.1, None, None), "must be >= 1"),
    (([4, 4], -1.0, None, None), "need rblock_tol >= 0"),
    (([4, 4], 0.1, -2, None), "need rblock_tol >= 0"),
])
def test_rblock_checks(lib, rblock, needle):
    d, obs = base()
    refused(lib, d, L.make_opts(rhat="block", rblock=rblock), needle)


def test_rblock_needs_sizes(lib):
    d, obs = base()
    o = L.make_opts()
    o.rhat = L.WC4D_RHAT_BLOCK
    refused(lib, d, o, "RHAT_BLOCK needs")


def test_null_problem_handles_are_refused(lib):
    """Entry points that take a problem refuse a null one (no dereference)."""
    n = None
    one = ctypes.c_void_p(1)       # never dereferenced: the null problem is checked first
    for rc in (lib.wc4d_apply_saddle(n, one, one), lib.wc4d_apply_precond(n, 0, one, one),
               lib.wc4d_solve(n, one, one, 0, L.WC4D_MEM_DEVICE, None), lib.wc4d_apply_fp32(n, 0, one, one),
               lib.wc4d_synthesize_rhs(n, one, one, L.WC4D_MEM_HOST, one), lib.wc4d_get_matrix(n, 0, one),
               lib.wc4d_precond_load(n, b"x"), lib.wc4d_precond_set_net(n, 32, one, 1)):
        assert rc == L.WC4D_ERR_ARG, lib.wc4d_last_error()
    nn = ctypes.c_int64()
    i = ctypes.c_int32()
    assert lib.wc4d_problem_dims(n, ctypes.byref(nn), ctypes.byref(i), ctypes.byref(i), ctypes.byref(i)) == \
        L.WC4D_ERR_ARG
    assert lib.wc4d_rhat_param(n) == 0.0
    lib.wc4d_destroy(n)            # a no-op
    lib.wc4d_default_opts(None)    # no-ops
    lib.wc4d_default_train_opts(None)


def test_batch_and_stats_arguments(lib):
    assert lib.wc4d_solve_batch(None, 1, None, None, 0, L.WC4D_MEM_DEVICE, 1, None) == L.WC4D_ERR_ARG
    assert lib.wc4d_get_stats(None) == L.WC4D_ERR_ARG
    st = L.Stats()
    lib.wc4d_reset_stats()
    assert lib.wc4d_get_stats(ctypes.byref(st)) == L.WC4D_OK
    assert st.launches == 0 and st.gemm_launches == 0


@pytest.mark.parametrize("basis, kw, needle", [
    (7, dict(), "basis_bytes must be 0, 6 or 8"),
    (6, dict(precision="fp64"), "basis_bytes 6 needs GMRES"),
    (6, dict(precision="ozaki", krylov="minres", precond="PD"), "basis_bytes 6 needs GMRES"),
    (6, dict(precision="ozaki", tol=1e-8), "needs tol >= 1e-7"),
])
def test_basis_bytes_checks(lib, basis, kw, needle):
    """The 6-byte Arnoldi basis (FP32 high + BF16 low part) is an option of
    the delayed-CGS2 GMRES only, at tolerances its rounding allows."""
    d, _ = base()
    args = dict(precond="PI", k=1, tol=1e-6)
    args.update(kw)
    o = L.make_opts(basis_bytes=basis, **args)
    refused(lib, d, o, needle)


def test_toeplitz_gemv_checks(lib):
    """toeplitz_gemv takes WC4D_TOEPLITZ_AUTO (0) or WC4D_TOEPLITZ_OFF (1)."""
    d, _ = base()
    for bad in (2, -1):
        o = L.make_opts(precond="PI", k=1, precision="ozaki", toeplitz_gemv=bad)
        refused(lib, d, o, "toeplitz_gemv must be")
