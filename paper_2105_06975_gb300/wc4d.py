"""Python binding of the wc4d C ABI (``include/wc4d.h``).

Argument marshalling only: every step of the solve runs in the CUDA library.
The library must be built (``paper_2105_06975_gb300.build.build()``); loading
fails loudly when it is missing -- there is no CPU fallback.

Functions keep the C names (``wc4d_setup_problem``, ``wc4d_apply_saddle``,
``wc4d_apply_precond``, ``wc4d_solve`` ...).  ``Problem`` is a small helper
that builds the descriptor from numpy arrays or workload parameters and
passes torch tensors' device pointers and the current torch CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

# ---------------------------------------------------------------- constants
WC4D_OK = 0
WC4D_ERR_ARG = 1
WC4D_ERR_NOT_SPD = 2
WC4D_ERR_NONFINITE = 3
WC4D_ERR_BREAKDOWN = 4
WC4D_ERR_MAXIT = 5
WC4D_ERR_TIMEOUT = 6
WC4D_ERR_CUDA = 7
WC4D_ERR_NOMEM = 8
WC4D_ERR_IO = 9

WC4D_MODEL_STENCIL3 = 0
WC4D_MODEL_BANDED = 1
WC4D_COV_DENSE = 0
WC4D_COV_SOAR = 1
WC4D_COV_MSOAR = 2
WC4D_MEM_HOST = 0
WC4D_MEM_DEVICE = 1
WC4D_PRECOND_PD = 0
WC4D_PRECOND_PI = 1
WC4D_RHAT_EXACT = 0
WC4D_RHAT_RR = 1
WC4D_RHAT_ME = 2
WC4D_RHAT_DIAG = 3
WC4D_RHAT_BLOCK = 4
WC4D_LHAT_LM = 0
WC4D_LHAT_I = 1
WC4D_SHAT_PAPER = 0
WC4D_SHAT_EXACT = 1
WC4D_SHAT_LEARNED = 2
WC4D_DHAT_EXACT = 0
WC4D_DHAT_SHIFT = 1
WC4D_KRYLOV_MINRES = 0
WC4D_KRYLOV_GMRES = 1
WC4D_KRYLOV_FGMRES = 2
WC4D_PREC_FP64 = 0
WC4D_PREC_MIXED = 1
WC4D_PREC_DF32 = 2
WC4D_PREC_DF32_P32 = 3
WC4D_PREC_OZAKI = 4
WC4D_COVPROD_DENSE = 0
WC4D_COVPROD_FFT = 1
WC4D_TOEPLITZ_AUTO = 0
WC4D_TOEPLITZ_OFF = 1

RHAT = {"exact": WC4D_RHAT_EXACT, "rr": WC4D_RHAT_RR, "me": WC4D_RHAT_ME, "diag": WC4D_RHAT_DIAG,
        "block": WC4D_RHAT_BLOCK}
LHAT = {"lm": WC4D_LHAT_LM, "i": WC4D_LHAT_I}
PRECOND = {"PD": WC4D_PRECOND_PD, "PI": WC4D_PRECOND_PI}
KRYLOV = {"minres": WC4D_KRYLOV_MINRES, "gmres": WC4D_KRYLOV_GMRES, "fgmres": WC4D_KRYLOV_FGMRES}

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)


class ProblemDesc(ctypes.Structure):
    _fields_ = [("s", ctypes.c_int32), ("N", ctypes.c_int32), ("p", ctypes.c_int32),
                ("model_kind", ctypes.c_int32), ("stencil", ctypes.c_double * 3),
                ("band_lo", ctypes.c_int32), ("band_hi", ctypes.c_int32), ("bands", ctypes.c_void_p),
                ("obs_idx", ctypes.c_void_p), ("cov_kind", ctypes.c_int32),
                ("B", ctypes.c_void_p), ("Q", ctypes.c_void_p), ("R", ctypes.c_void_p),
                ("soar_b", ctypes.c_double * 2), ("soar_q", ctypes.c_double * 2), ("soar_r", ctypes.c_double * 2),
                ("mem_kind", ctypes.c_int32), ("msoar_b", ctypes.c_double * 3), ("msoar_q", ctypes.c_double * 3),
                ("msoar_psi", ctypes.c_double * 2), ("p_t", ctypes.POINTER(ctypes.c_int32))]


class SolveOpts(ctypes.Structure):
    _fields_ = [("precond", ctypes.c_int32), ("k", ctypes.c_int32), ("rhat", ctypes.c_int32),
                ("kappa_max", ctypes.c_double), ("shat", ctypes.c_int32), ("dhat", ctypes.c_int32),
                ("dhat_delta", ctypes.c_double), ("krylov", ctypes.c_int32), ("tol", ctypes.c_double),
                ("maxit", ctypes.c_int32), ("precision", ctypes.c_int32), ("inner_iters", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("lhat", ctypes.c_int32), ("rblock_count", ctypes.c_int32),
                ("rblock_sizes", ctypes.POINTER(ctypes.c_int32)), ("rblock_tol", ctypes.c_double),
                ("rblock_maxsize", ctypes.c_int32), ("rblock_numproc", ctypes.c_int32),
                ("covprod", ctypes.c_int32), ("prec_digits", ctypes.c_int32), ("rinv_explicit", ctypes.c_int32),
                ("basis_bytes", ctypes.c_int32), ("toeplitz_gemv", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("inner_iters", ctypes.c_int32),
                ("precond_fallback", ctypes.c_int32),
                ("relres_true", ctypes.c_double), ("relres_est", ctypes.c_double), ("ms", ctypes.c_double),
                ("n_apply_A", ctypes.c_int64), ("n_apply_P", ctypes.c_int64),
                ("n_cov", ctypes.c_int64), ("n_M", ctypes.c_int64), ("n_trsm", ctypes.c_int64),
                ("n_R", ctypes.c_int64), ("n_D", ctypes.c_int64), ("n_Dhat_inv", ctypes.c_int64),
                ("n_Rhat_inv", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("gemm_ms", ctypes.c_double), ("gemm_flops", ctypes.c_double),
                ("gemm_launches", ctypes.c_int64), ("orth_ms", ctypes.c_double), ("orth_bytes", ctypes.c_double),
                ("orth_launches", ctypes.c_int64), ("gemm32_ms", ctypes.c_double), ("gemm32_flops", ctypes.c_double),
                ("gemm32_launches", ctypes.c_int64), ("gemmdf_ms", ctypes.c_double),
                ("gemmdf_flops", ctypes.c_double), ("gemmdf_launches", ctypes.c_int64),
                ("gemmtc_ms", ctypes.c_double), ("gemmtc_flops", ctypes.c_double),
                ("gemmtc_bytes", ctypes.c_double), ("gemmtc_mma_flops", ctypes.c_double),
                ("gemmtc_launches", ctypes.c_int64), ("gemmtc_alg_bytes", ctypes.c_double),
                ("circ_ms", ctypes.c_double), ("circ_flops", ctypes.c_double),
                ("circ_bytes", ctypes.c_double), ("circ_launches", ctypes.c_int64), ("pt_ms", ctypes.c_double),
                ("pt_bytes", ctypes.c_double), ("pt_launches", ctypes.c_int64),
                ("orth_moved_bytes", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class TrainOpts(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_int32), ("hidden", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("epochs", ctypes.c_int32), ("lr", ctypes.c_double), ("val_frac", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("loss", ctypes.c_int32)]


WC4D_LOSS_ERROR = 0
WC4D_LOSS_RESIDUAL = 1


class TrainReport(ctypes.Structure):
    _fields_ = [("loss_first", ctypes.c_double), ("loss_last", ctypes.c_double),
                ("val_err_learned", ctypes.c_double), ("val_err_plain", ctypes.c_double),
                ("kept", ctypes.c_int32), ("pairs_train", ctypes.c_int32),
                ("gen_ms", ctypes.c_double), ("train_ms", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class L96Params(ctypes.Structure):
    _fields_ = [("forcing", ctypes.c_double), ("dt", ctypes.c_double), ("steps_per_obs", ctypes.c_int32),
                ("outer_loops", ctypes.c_int32)]


# names and signatures of every entry point declared in include/wc4d.h
SIGNATURES = {
    "wc4d_default_opts": (None, [ctypes.POINTER(SolveOpts)]),
    "wc4d_setup_problem": (ctypes.c_int, [ctypes.POINTER(ProblemDesc), ctypes.POINTER(SolveOpts), ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_void_p)]),
    "wc4d_apply_saddle": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "wc4d_apply_precond": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "wc4d_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                  ctypes.POINTER(Info)]),
    "wc4d_status": (ctypes.c_int, [ctypes.c_void_p]),
    "wc4d_set_wait_limit_ns": (None, [ctypes.c_uint64]),
    "wc4d_apply_fp32": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "wc4d_solve_batch": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(Info)]),
    "wc4d_synthesize_rhs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                           ctypes.c_void_p]),
    "wc4d_l96_gauss_newton": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(L96Params), ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.POINTER(Info)]),
    "wc4d_l96_linearize": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(L96Params), ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "wc4d_problem_dims": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), _ip, _ip, _ip]),
    "wc4d_get_matrix": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "wc4d_rhat_param": (ctypes.c_double, [ctypes.c_void_p]),
    "wc4d_set_profiling": (None, [ctypes.c_int32]),
    "wc4d_reset_stats": (None, []),
    "wc4d_get_stats": (ctypes.c_int, [ctypes.POINTER(Stats)]),
    "wc4d_apply_saddle_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                 ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_void_p]),
    "wc4d_default_train_opts": (None, [ctypes.POINTER(TrainOpts)]),
    "wc4d_precond_train": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(TrainOpts), ctypes.c_char_p,
                                          ctypes.POINTER(TrainReport)]),
    "wc4d_precond_load": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "wc4d_precond_set_net": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32]),
    "wc4d_net_grad": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                     ctypes.c_void_p]),
    "wc4d_net_nparams": (ctypes.c_int64, [ctypes.c_int32, ctypes.c_int32]),
    "wc4d_destroy": (None, [ctypes.c_void_p]),
    "wc4d_last_error": (ctypes.c_char_p, []),
}

_LIB = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libwc4d.so (building it first if allowed).  Raises if it cannot."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"wc4d CUDA library not built: {path}")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


class WC4DError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"wc4d error {code}: {msg}")
        self.code = code


def _check(code):
    if code != WC4D_OK:
        raise WC4DError(code, load().wc4d_last_error().decode())
    return code


# ------------------------------------------------------------ thin wrappers
def wc4d_default_opts() -> SolveOpts:
    o = SolveOpts()
    load().wc4d_default_opts(ctypes.byref(o))
    return o


def wc4d_setup_problem(desc: ProblemDesc, opts: SolveOpts, stream: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().wc4d_setup_problem(ctypes.byref(desc), ctypes.byref(opts), ctypes.c_void_p(stream),
                                     ctypes.byref(h)))
    return h


def wc4d_apply_saddle(h, v_ptr: int, out_ptr: int) -> None:
    _check(load().wc4d_apply_saddle(h, ctypes.c_void_p(v_ptr), ctypes.c_void_p(out_ptr)))


def wc4d_apply_precond(h, which: int, v_ptr: int, out_ptr: int) -> None:
    _check(load().wc4d_apply_precond(h, which, ctypes.c_void_p(v_ptr), ctypes.c_void_p(out_ptr)))


def wc4d_status(h, raise_on_error=True) -> int:
    """Synchronise the problem's stream and report (then clear) a bounded
    device wait that gave up since the last check (WC4D_ERR_TIMEOUT)."""
    code = load().wc4d_status(h)
    if raise_on_error:
        _check(code)
    return code


def wc4d_set_wait_limit_ns(ns: int) -> None:
    load().wc4d_set_wait_limit_ns(int(ns))


def wc4d_solve(h, rhs_ptr: int, x_ptr: int, use_x0: bool, mem_kind: int, raise_on_error=True) -> Info:
    info = Info()
    code = load().wc4d_solve(h, ctypes.c_void_p(rhs_ptr), ctypes.c_void_p(x_ptr), int(use_x0), mem_kind,
                             ctypes.byref(info))
    if raise_on_error and code not in (WC4D_OK, WC4D_ERR_MAXIT):
        _check(code)
    info.status = code
    return info


def wc4d_solve_batch(handles, rhs_ptrs, x_ptrs, use_x0: bool, mem_kind: int, workers: int = 0,
                     raise_on_error=True):
    """Solve len(handles) independent problems concurrently; returns (code, [Info])."""
    cnt = len(handles)
    H = (ctypes.c_void_p * max(cnt, 1))(*handles)
    R = (ctypes.c_void_p * max(cnt, 1))(*rhs_ptrs)
    X = (ctypes.c_void_p * max(cnt, 1))(*x_ptrs)
    infos = (Info * max(cnt, 1))()
    code = load().wc4d_solve_batch(H, cnt, R, X, int(use_x0), mem_kind, int(workers), infos)
    if raise_on_error and code not in (WC4D_OK, WC4D_ERR_MAXIT):
        _check(code)
    return code, [infos[i] for i in range(cnt)]


def solve_batch(problems, rhs_list, x_list=None, use_x0=False, workers=0):
    """Batched solve of Problem objects: rhs_list entries are numpy arrays (host
    path) or CUDA tensors (device path), all of one kind."""
    import numpy as _np
    host = isinstance(rhs_list[0], _np.ndarray)
    if host:
        rhs_list = [_np.ascontiguousarray(r, dtype=_np.float64) for r in rhs_list]
        if x_list is None:
            x_list = [_np.zeros_like(r) for r in rhs_list]
        rp = [r.ctypes.data for r in rhs_list]
        xp = [x.ctypes.data for x in x_list]
    else:
        import torch as _torch
        if x_list is None:
            x_list = [_torch.zeros_like(r) for r in rhs_list]
        rp = [r.data_ptr() for r in rhs_list]
        xp = [x.data_ptr() for x in x_list]
    code, infos = wc4d_solve_batch([p.h for p in problems], rp, xp, use_x0,
                                   WC4D_MEM_HOST if host else WC4D_MEM_DEVICE, workers)
    return x_list, infos, code


def net_nparams(C: int, hidden: int) -> int:
    return int(load().wc4d_net_nparams(int(C), int(hidden)))


def net_grad(C, hidden, s, params, yn, tn):
    """Library (device) mean loss and parameter gradients of the learned net on
    host samples yn, tn of shape [B, C, s]."""
    params = np.ascontiguousarray(params, dtype=np.float32)
    yn = np.ascontiguousarray(yn, dtype=np.float32)
    tn = np.ascontiguousarray(tn, dtype=np.float32)
    B = yn.shape[0]
    grads = np.zeros_like(params)
    loss = ctypes.c_double(0.0)
    _check(load().wc4d_net_grad(int(C), int(hidden), int(s), int(B), ctypes.c_void_p(params.ctypes.data),
                                ctypes.c_void_p(yn.ctypes.data), ctypes.c_void_p(tn.ctypes.data),
                                ctypes.byref(loss), ctypes.c_void_p(grads.ctypes.data)))
    return loss.value, grads


def wc4d_apply_fp32(h, which: int, v_ptr: int, out_ptr: int) -> None:
    _check(load().wc4d_apply_fp32(h, which, ctypes.c_void_p(v_ptr), ctypes.c_void_p(out_ptr)))


def wc4d_synthesize_rhs(h, zb_ptr: int, zr_ptr: int, mem_kind: int, rhs_ptr: int) -> None:
    _check(load().wc4d_synthesize_rhs(h, ctypes.c_void_p(zb_ptr), ctypes.c_void_p(zr_ptr), mem_kind,
                                      ctypes.c_void_p(rhs_ptr)))


def wc4d_l96_gauss_newton(h, forcing, dt, steps, loops, xb_ptr, y_ptr, traj_ptr, init_background, mem_kind):
    prm = L96Params(float(forcing), float(dt), int(steps), int(loops))
    infos = (Info * int(loops))()
    code = load().wc4d_l96_gauss_newton(h, ctypes.byref(prm), ctypes.c_void_p(xb_ptr), ctypes.c_void_p(y_ptr),
                                        ctypes.c_void_p(traj_ptr), int(init_background), mem_kind, infos)
    if code not in (WC4D_OK, WC4D_ERR_MAXIT):
        _check(code)
    return code, [infos[i] for i in range(int(loops))]


def wc4d_problem_dims(h):
    n = ctypes.c_int64()
    s, N, p = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().wc4d_problem_dims(h, ctypes.byref(n), ctypes.byref(s), ctypes.byref(N), ctypes.byref(p)))
    return n.value, s.value, N.value, p.value


def wc4d_get_matrix(h, which: int, dst_ptr: int) -> None:
    _check(load().wc4d_get_matrix(h, which, ctypes.c_void_p(dst_ptr)))


def wc4d_rhat_param(h) -> float:
    return load().wc4d_rhat_param(h)


def wc4d_set_profiling(enable: bool) -> None:
    load().wc4d_set_profiling(int(bool(enable)))


def wc4d_reset_stats() -> None:
    load().wc4d_reset_stats()


def wc4d_get_stats() -> Stats:
    st = Stats()
    _check(load().wc4d_get_stats(ctypes.byref(st)))
    return st


def wc4d_apply_saddle_noalloc(s, N, p, stencil, obs_ptr, B_ptr, Q_ptr, R_ptr, v_ptr, out_ptr, stream=0) -> None:
    """A v from caller-owned device arrays without any device allocation
    (see the header for the limits and the shared scratch array)."""
    c = (ctypes.c_double * 3)(*[float(x) for x in stencil])
    _check(load().wc4d_apply_saddle_noalloc(int(s), int(N), int(p), c, ctypes.c_void_p(obs_ptr),
                                            ctypes.c_void_p(B_ptr), ctypes.c_void_p(Q_ptr), ctypes.c_void_p(R_ptr),
                                            ctypes.c_void_p(v_ptr), ctypes.c_void_p(out_ptr),
                                            ctypes.c_void_p(stream)))


def wc4d_destroy(h) -> None:
    load().wc4d_destroy(h)


def wc4d_last_error() -> str:
    return load().wc4d_last_error().decode()


# -------------------------------------------------------------- convenience
def make_opts(precond="PI", k=1, rhat="exact", kappa_max=100.0, shat="paper", dhat="exact", dhat_delta=0.01,
              krylov=None, tol=1e-6, maxit=1000, precision="fp64", inner_iters=20, check_every=4, lhat="lm",
              rblock=None, covprod="dense", prec_digits=0, rinv_explicit=False, basis_bytes=0,
              toeplitz_gemv=WC4D_TOEPLITZ_AUTO) -> SolveOpts:
    """``rblock`` = (channel block sizes, tol, maxsize, numproc) for rhat="block"
    (Alg. 3; maxsize / numproc None or 0 switch their rule off)."""
    o = wc4d_default_opts()
    o.lhat = LHAT[lhat]
    if rblock is not None:
        sizes, btol, maxsize, numproc = rblock
        arr = (ctypes.c_int32 * len(sizes))(*[int(x) for x in sizes])
        o._rblock_keep = arr          # the library reads the sizes during setup
        o.rblock_count = len(sizes)
        o.rblock_sizes = ctypes.cast(arr, ctypes.POINTER(ctypes.c_int32))
        o.rblock_tol = float(btol)
        o.rblock_maxsize = int(maxsize or 0)
        o.rblock_numproc = int(numproc or 0)
    o.precond = PRECOND[precond]
    o.k = int(k)
    o.rhat = RHAT[rhat]
    o.kappa_max = float(kappa_max)
    o.shat = {"paper": WC4D_SHAT_PAPER, "exact": WC4D_SHAT_EXACT, "learned": WC4D_SHAT_LEARNED}[shat]
    o.dhat = WC4D_DHAT_SHIFT if dhat in ("rr", "shift") else WC4D_DHAT_EXACT
    o.dhat_delta = float(dhat_delta)
    if krylov is None:
        krylov = "fgmres" if precision == "mixed" else ("minres" if precond == "PD" else "gmres")
    o.krylov = KRYLOV[krylov]
    o.tol = float(tol)
    o.maxit = int(maxit)
    o.precision = {"fp64": WC4D_PREC_FP64, "mixed": WC4D_PREC_MIXED, "df32": WC4D_PREC_DF32,
                   "df32p32": WC4D_PREC_DF32_P32, "ozaki": WC4D_PREC_OZAKI}[precision]
    o.inner_iters = int(inner_iters)
    o.check_every = int(check_every)
    o.covprod = {"dense": WC4D_COVPROD_DENSE, "fft": WC4D_COVPROD_FFT}[covprod]
    o.prec_digits = int(prec_digits)
    o.rinv_explicit = int(bool(rinv_explicit))
    o.basis_bytes = int(basis_bytes)
    o.toeplitz_gemv = int(toeplitz_gemv)
    return o


class Problem:
    """Owns a wc4d problem handle.  Host arrays are passed with mem_kind=HOST
    and copied by the library; the handle is freed by ``close()``/``__del__``."""

    def __init__(self, s, N, p, obs_idx, opts: SolveOpts, *, stencil=None, bands=None, band_lo=0, band_hi=0,
                 banded=False, B=None, Q=None, R=None, soar_b=None, soar_q=None, soar_r=None,
                 stream: Optional[int] = None, obs_list=None, msoar=None):
        """``obs_list``: per-time observation sets (N+1 sorted index arrays);
        then ``p`` and ``obs_idx`` are ignored and a dense ``R`` is a list of
        the N+1 blocks R_i."""
        import torch
        d = ProblemDesc()
        keep = []

        def host(a, dtype):
            a = np.ascontiguousarray(a, dtype=dtype)
            keep.append(a)
            return a.ctypes.data
        if obs_list is not None:
            pt = np.array([len(o) for o in obs_list], dtype=np.int32)
            keep.append(pt)
            d.p_t = pt.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            p = int(pt.sum())
            obs_idx = np.concatenate([np.asarray(o, dtype=np.int32) for o in obs_list])
            if R is not None and not isinstance(R, np.ndarray):
                R = np.concatenate([np.ascontiguousarray(Ri, dtype=np.float64).ravel() for Ri in R])
        d.s, d.N, d.p = int(s), int(N), int(p)
        d.obs_idx = host(obs_idx, np.int32)
        if bands is not None or banded:
            d.model_kind = WC4D_MODEL_BANDED
            d.bands = host(bands, np.float64) if bands is not None else None
            d.band_lo, d.band_hi = int(band_lo), int(band_hi)
        else:
            d.model_kind = WC4D_MODEL_STENCIL3
            d.stencil[:] = [float(c) for c in stencil]
        if msoar is not None:
            # banded circulant B, Q: ((amp, L, maxval) of B, of Q, (psi_B, psi_Q)); R dense or SOAR
            d.cov_kind = WC4D_COV_MSOAR
            d.msoar_b[:] = [float(x) for x in msoar[0]]
            d.msoar_q[:] = [float(x) for x in msoar[1]]
            d.msoar_psi[:] = [float(x) for x in msoar[2]]
            if R is not None:
                d.R = host(R, np.float64)
            else:
                d.soar_r[:] = list(soar_r)
        elif B is not None:
            d.cov_kind = WC4D_COV_DENSE
            # column-major == row-major for the symmetric covariances
            d.B, d.Q, d.R = host(B, np.float64), host(Q, np.float64), host(R, np.float64)
        else:
            d.cov_kind = WC4D_COV_SOAR
            d.soar_b[:] = list(soar_b)
            d.soar_q[:] = list(soar_q)
            d.soar_r[:] = list(soar_r)
        d.mem_kind = WC4D_MEM_HOST
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        self.opts = opts
        self.h = wc4d_setup_problem(d, opts, stream)
        self.n, self.s, self.N, self.p = wc4d_problem_dims(self.h)

    @classmethod
    def from_workload(cls, w, dr, opts: SolveOpts, dense=False, **kw):
        """Build from a ``workload.Workload`` and its draws; SOAR covariances
        are generated by the library unless ``dense`` arrays are given in kw."""
        c = w.stencil()
        if dense:
            return cls(w.s, w.N, w.p, dr.obs_idx, opts, stencil=c, **kw)
        if w.obs_per_time and "obs_list" not in kw:
            kw["obs_list"] = dr.extra["obs_list"]
        return cls(w.s, w.N, w.p, dr.obs_idx, opts, stencil=kw.pop("stencil", c), soar_b=w.soar_b,
                   soar_q=w.soar_q, soar_r=w.soar_r, **kw)

    def apply_saddle(self, v, out=None):
        import torch
        out = torch.empty_like(v) if out is None else out
        wc4d_apply_saddle(self.h, v.data_ptr(), out.data_ptr())
        return out

    def apply_precond(self, which, v, out=None):
        import torch
        out = torch.empty_like(v) if out is None else out
        wc4d_apply_precond(self.h, PRECOND[which] if isinstance(which, str) else which, v.data_ptr(),
                           out.data_ptr())
        return out

    def solve(self, rhs, x=None, use_x0=False):
        """rhs/x: torch CUDA tensors (device path) or numpy arrays (host path)."""
        if isinstance(rhs, np.ndarray):
            rhs = np.ascontiguousarray(rhs, dtype=np.float64)
            x = np.zeros_like(rhs) if x is None else x
            info = wc4d_solve(self.h, rhs.ctypes.data, x.ctypes.data, use_x0, WC4D_MEM_HOST)
            return x, info
        import torch
        x = torch.zeros_like(rhs) if x is None else x
        info = wc4d_solve(self.h, rhs.data_ptr(), x.data_ptr(), use_x0, WC4D_MEM_DEVICE)
        return x, info

    def apply_fp32(self, which, v):
        """which: "A", "PD" or "PI"; v: float32 CUDA tensor."""
        import torch
        out = torch.empty_like(v)
        wc4d_apply_fp32(self.h, {"A": 0, "PD": 1, "PI": 2}[which], v.data_ptr(), out.data_ptr())
        return out

    def synthesize_rhs(self, dr):
        """Device-built (b, d, 0) from the draws' z_b, z_r (linear models)."""
        import torch
        zb = torch.from_numpy(np.ascontiguousarray(dr.z_b, dtype=np.float64)).cuda()
        zr = torch.from_numpy(np.ascontiguousarray(dr.z_r, dtype=np.float64)).cuda()
        rhs = torch.empty(self.n, dtype=torch.float64, device="cuda")
        wc4d_synthesize_rhs(self.h, zb.data_ptr(), zr.data_ptr(), WC4D_MEM_DEVICE, rhs.data_ptr())
        return rhs

    def l96_gauss_newton(self, forcing, dt, steps, loops, xb, y, traj=None):
        """Host arrays in, final trajectory (N+1, s) and per-loop Info out."""
        xb = np.ascontiguousarray(xb, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        out = np.zeros((self.N + 1, self.s)) if traj is None else np.ascontiguousarray(traj, dtype=np.float64).copy()
        code, infos = wc4d_l96_gauss_newton(self.h, forcing, dt, steps, loops, xb.ctypes.data, y.ctypes.data,
                                            out.ctypes.data, traj is None, WC4D_MEM_HOST)
        return out, infos, code

    def l96_linearize(self, forcing, dt, steps, xb, y, traj):
        """Rebuild the banded M_t about traj; return the right-hand side (host)."""
        xb, y, traj = (np.ascontiguousarray(a, dtype=np.float64) for a in (xb, y, traj))
        rhs = np.zeros(self.n)
        prm = L96Params(float(forcing), float(dt), int(steps), 0)
        _check(load().wc4d_l96_linearize(self.h, ctypes.byref(prm), ctypes.c_void_p(xb.ctypes.data),
                                         ctypes.c_void_p(y.ctypes.data), ctypes.c_void_p(traj.ctypes.data),
                                         WC4D_MEM_HOST, ctypes.c_void_p(rhs.ctypes.data)))
        return rhs

    def precond_train(self, pairs=50000, hidden=32, batch=64, epochs=4, lr=1e-3, val_frac=0.05, seed=1,
                      ckpt_path=None, loss="error"):
        """Train the learned Schur block on the device; returns the TrainReport.
        loss: "error" (|z - S^-1 r| / |S^-1 r|) or "residual" (|S z - r| / |r|)."""
        o = TrainOpts()
        load().wc4d_default_train_opts(ctypes.byref(o))
        o.pairs, o.hidden, o.batch, o.epochs = int(pairs), int(hidden), int(batch), int(epochs)
        o.lr, o.val_frac, o.seed = float(lr), float(val_frac), int(seed)
        o.loss = {"error": WC4D_LOSS_ERROR, "residual": WC4D_LOSS_RESIDUAL}[loss]
        rep = TrainReport()
        path = ckpt_path.encode() if ckpt_path else None
        _check(load().wc4d_precond_train(self.h, ctypes.byref(o), path, ctypes.byref(rep)))
        return rep

    def precond_load(self, ckpt_path):
        _check(load().wc4d_precond_load(self.h, ckpt_path.encode()))

    def precond_set_net(self, hidden, params, active=True):
        w = np.ascontiguousarray(params, dtype=np.float32)
        _check(load().wc4d_precond_set_net(self.h, int(hidden), ctypes.c_void_p(w.ctypes.data), int(active)))

    def matrix(self, which):
        import torch
        m = self.s if which in (0, 1) else self.p
        out = torch.empty((m, m), dtype=torch.float64, device="cuda")
        wc4d_get_matrix(self.h, which, out.data_ptr())
        return out

    def rhat_param(self):
        return wc4d_rhat_param(self.h)

    def close(self):
        if getattr(self, "h", None):
            wc4d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
