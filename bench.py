#!/usr/bin/env python
"""Benchmark: saddle-point solves per second of weak-constraint 4D-Var.

One step = one pass of the whole method over one assimilation window: build
the problem on the device (SOAR covariances, Rhat, FP64 Cholesky factors and
their inverses, GEMM schedules) and solve the saddle-point system to a true
relative residual of 1e-6 (Sec. 6.2 / Sec. 7).  The window is the scale
advection-diffusion workload: s=2048, N=64 (65 time levels), p=1024 randomly
observed points, SOAR B/Q/R, n = 332,800 unknowns.  Its right-hand side is
built on the device before timing (inputs resident in HBM).

Launch: ``python bench.py --gpus N --steps K --warmup W`` (N > 1 under
torch.distributed.run, one window per rank, weak scaling, no data-path
collective).  ``--impl reference`` times the FP64 CPU oracle on the host
cores: each timed step is one full solve of the same window; steps stop early
once the next would overrun ``--ref-budget-s``, and ``steps`` reports the
solves that ran.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "saddle solves/s to rel-res 1e-6 (chosen vs plain FP64 GPU); % HBM roofline"
UNIT = "solves/s"
# FP64 FMA peak derived from unit counts and clock: 152 SMs x 4 FP64 flop/clk
# x 2.07 GHz (the recipe's nominal 1.25 TFLOP/s; a project micro-benchmark
# measured 1.196 TFLOP/s at 1.995 GHz)
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--precond", default="PI")
    ap.add_argument("--k", type=int, default=4)
    ap.add_argument("--rhat", default="exact")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--maxit", type=int, default=1000, help="Krylov iteration cap (workspace size)")
    ap.add_argument("--inner", type=int, default=20, help="inner FP32 GMRES steps per outer FGMRES step")
    ap.add_argument("--mixed", action="store_true", help="also time the nested FP32-inner mode")
    ap.add_argument("--chosen", default="ozaki_rinv_b6", choices=["fp64", "df32", "df32p32", "mixed", "ozaki", "fp64_fft",
                                                          "df32_fft", "ozaki_fft", "ozaki_rinv",
                                                          "ozaki_rinv_b6", "ozaki_fft_rinv_b6"])
    ap.add_argument("--precision", default="ozaki", choices=["df32", "ozaki"],
                    help="product precision of the batched and learned workloads")
    ap.add_argument("--rinv", action="store_true",
                    help="batched workload: Rhat^-1 as one product with the explicit inverse")
    ap.add_argument("--modes", default=None, help="comma list of modes to time (default: fp64,chosen)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-comparisons", action="store_true",
                    help="skip the P_D + MINRES and circulant-FFT comparison solves of the default line")
    ap.add_argument("--ref-budget-s", type=float, default=240.0,
                    help="reference arm: time budget for its timed full oracle solves (stops early)")
    ap.add_argument("--no-clocks", action="store_true", help="do not sample nvidia-smi (profiler runs)")
    ap.add_argument("--workload", default="scale", choices=["scale", "batch", "learned", "profile", "heat"],
                    help="scale: one s=2048 N=64 window (default line); batch: independent uneven windows; "
                         "learned: learned Schur block vs the plain P_D (s=1024 N=32); heat: the heat equation at "
                         "s=50,000 N=5 p=12,500 with banded B, Q; profile: a small fixed "
                         "run of the hot kernels at the scale sizes for ncu captures (products, then one "
                         "solve of --maxit GMRES steps)")
    ap.add_argument("--pairs", type=int, default=50000, help="training pairs of the learned workload")
    ap.add_argument("--epochs", type=int, default=4, help="training epochs of the learned workload")
    ap.add_argument("--loss", default="error", choices=["error", "residual"],
                    help="learned workload: train on the Schur-solve error or the preconditioned residual")
    ap.add_argument("--batch", type=int, default=256, help="windows in the batched workload")
    ap.add_argument("--batch-maxit", type=int, default=300, help="Krylov cap per batched window")
    ap.add_argument("--workers", type=int, default=8, help="host workers / CUDA streams of the batched solve")
    ap.add_argument("--check-every", type=int, default=4, help="Krylov steps between convergence polls")
    return ap.parse_args()


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def dist_info():
    from paper_2105_06975_gb300.ranks import dist_info as _di
    return _di()


# --------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ CPU oracle
def host_threads():
    """Threads the oracle's numpy/BLAS work runs on: the BLAS thread-count
    variables when set, else the cores this process may run on."""
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        try:
            return max(1, int(os.environ[var]))
        except (KeyError, ValueError):
            pass
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def oracle_solve(args, w, dr, maxit=1000, tol=1e-6):
    """One full solve by the FP64 oracle, timed on the host cores: problem
    build + Rhat factor + the Krylov solve to ``tol`` (the GPU solve's
    stopping rule).  With ``tol=0`` and a small ``maxit`` it is a short
    untimed warm-up (BLAS thread pool, page-in)."""
    from oracle import krylov, problem as prb, saddle as sd
    t0 = time.perf_counter()
    prob, obs, rhs = prb.linear_case(w, dr)
    P = sd.Preconditioner(prob, sd.PrecondOptions(kind=args.precond, k=args.k, rhat=args.rhat))
    t1 = time.perf_counter()
    if args.precond == "PD":
        r = krylov.minres(prob.A_apply, P.apply, rhs, tol=tol, maxit=maxit)
    else:
        r = krylov.gmres(prob.A_apply, P.apply, rhs, tol=tol, maxit=maxit)
    t2 = time.perf_counter()
    name = "MINRES" if args.precond == "PD" else "GMRES"
    cores = host_threads()
    return {"value": 1.0 / (t2 - t0), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"one full solve of the same window: problem build + Rhat factor ({t1 - t0:.2f} s) + "
                       f"{r.iters} {name} iterations to true relative residual {r.relres_true:.3g} "
                       f"({t2 - t1:.2f} s); numpy FP64 on {cores} host threads"),
            "iterations": r.iters, "relres_true": r.relres_true, "converged": bool(r.converged),
            "t_total": t2 - t0}


def workload_config(args, w):
    return {"workload": f"advection-diffusion window s={w.s} N={w.N} p={w.p} (n={w.n}), SOAR B/Q/R",
            "s": w.s, "N": w.N, "p": w.p, "n": w.n, "precond": args.precond, "lhat": f"L_M({args.k})",
            "rhat": args.rhat, "krylov": "MINRES" if args.precond == "PD" else "GMRES (no restart)",
            "tol": 1e-6, "step": "device problem build (SOAR, Rhat, Cholesky, inverse factors) + solve",
            "l2": "flushed between steps (256 MiB write); matrices are rebuilt every step"}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    from paper_2105_06975_gb300 import workload as W
    w = W.SCALE
    dr = W.draws(w, args.seed)
    # warm-up steps are short untimed oracle runs (imports, BLAS threads,
    # page-in); every timed step is one full oracle solve (~13-30 s on 8-16
    # host cores at this size).  Steps stop early once the next one would not
    # fit in --ref-budget-s, and the line reports the solves that ran.
    for _ in range(args.warmup):
        oracle_solve(args, w, dr, maxit=2, tol=0.0)
    t_start = time.perf_counter()
    vals = []
    for _ in range(args.steps):
        elapsed = time.perf_counter() - t_start
        if vals and elapsed + vals[0]["t_total"] > args.ref_budget_s:
            break
        vals.append(oracle_solve(args, w, dr))
    wall = time.perf_counter() - t_start
    v = len(vals) / sum(x["t_total"] for x in vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": len(vals), "steps_requested": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args, w), "timed_wall_s": wall,
            "cpu_baseline": {**{k: vals[0][k] for k in ("unit", "cores", "kind", "iterations", "relres_true",
                                                        "converged")},
                             "value": v,
                             "sample": (f"{len(vals)} timed steps, each one full oracle solve ("
                                        + vals[0]["sample"] + ")"
                                        + (f"; stopped after {len(vals)} of {args.steps} requested steps to stay "
                                           f"within {args.ref_budget_s:.0f} s" if len(vals) < args.steps
                                           else ""))},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- GPU
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # FP32 FMA: 128/clk/SM (measured 74.4 TF at 1.995 GHz)
# double-float multiply-add = 12 FP32 lane operations (1 FMUL, 3 FFMA, 8 FADD; the
# paired FFMA2/FADD2 forms do two lanes per instruction but not more lanes per clock):
# FP64-equivalent peak of the FP32 pipe = 2 flop x 152 SM x 128 lanes x 2.07 GHz / 12
DF32_PEAK_TFLOPS = 2 * 152 * 128 * 2.07e9 / 12 / 1e12
MODE_DTYPE = {"fp64": "f64", "df32": "df32 products (2 x f32, ~48-bit) / f64 recurrences",
              "mixed": "f32 inner / df32-f64 outer",
              "ozaki": "bf16 digit products exact in f32 (47-bit operands as 7 digits) / df32 / f64 recurrences",
              "fp64_fft": "f64 (B, Q by f64 FFT)",
              "df32_fft": "f64 FFT for B, Q; df32 R-family products / f64 recurrences",
              "ozaki_fft": "f64 FFT for B, Q; bf16 digit products exact in f32 for the R family / df32 / f64 "
                           "recurrences",
              "ozaki_rinv": "bf16 digit products exact in f32 (47-bit operands as 7 digits) / df32 / f64 recurrences",
              "ozaki_rinv_b6": "bf16 digit products exact in f32 (47-bit operands as 7 digits) / f32+bf16 Arnoldi "
                               "basis / f64 recurrences",
              "ozaki_fft_rinv_b6": "df32 FFT for B, Q; bf16 digit products exact in f32 for the R family / f32+bf16 "
                                   "Arnoldi basis / f64 recurrences"}
MODE_DESC = {"fp64": "plain FP64: native DFMA products, FP64 GMRES",
             "df32": "FP64 GMRES; covariance / factor products in double-float on the FP32 pipe",
             "ozaki": "FP64 GMRES; multi-column covariance / factor products as exact BF16 digit products "
                      "on the tensor cores (tcgen05, TMEM accumulators), one-column products in double-float",
             "mixed": "FGMRES outer (double-float A, FP64 true residual) around FP32 inner GMRES({inner}) "
                      "preconditioned by FP32 {pc}",
             "fp64_fft": "plain FP64 with circulant B, Q (and Bhat^-1, Qhat^-1) by FP64 FFT",
             "df32_fft": "FP64 Krylov; circulant B, Q by FP64 FFT; R-family products in double-float",
             "ozaki_fft": "FP64 Krylov; circulant B, Q (and Bhat^-1, Qhat^-1) by FFT (cluster-split "
                          "four-step transform, double-float); multi-column R-family products as exact BF16 digit "
                          "products on tcgen05",
             "ozaki_rinv": "FP64 GMRES; multi-column covariance / factor products as exact BF16 digit products on "
                           "tcgen05; Rhat^-1 as one product with the explicit inverse W^T W (in the launch of "
                           "P_I's D c1)",
             "ozaki_rinv_b6": "FP64 GMRES; multi-column covariance / factor products as exact BF16 digit products "
                              "on tcgen05; Rhat^-1 as one product with the explicit inverse W^T W; Arnoldi basis "
                              "stored as FP32 high + BF16 low parts (6 B per entry, about 32 bits); B's one-column "
                              "products in double-float from its first row (B is symmetric Toeplitz)",
             "ozaki_fft_rinv_b6": "FP64 GMRES; circulant B, Q (and Bhat^-1, Qhat^-1) by double-float FFT (cluster-"
                                  "split four-step transform); R-family products as exact BF16 digit products on "
                                  "tcgen05 with the explicit Rhat^-1; 6-byte Arnoldi basis"}


# DRAM bytes per launch of gemm_streamk_df32_kernel, ncu dram__bytes_read.sum + dram__bytes_write.sum,
# mean over the three product launches of one GMRES step (P_I level 1, P_I level 2, A v) at the scale
# workload; captured on a GB300 (summary and command in profiles/gemm_streamk_df32__advdiff_s2048_N64.md).
# Valid while that kernel is unchanged.
GEMM_DF32_TRAFFIC_BYTES = 53.3e6
# DRAM bytes (read + write) over algorithmic bytes of one captured launch, for kernels whose
# bytes per launch vary with the launch (Arnoldi step j, product type): traffic per launch =
# ratio x the live algorithmic bytes per launch.  Captured on a GB300 with
# `bench.py --workload profile --maxit 110` (summaries and commands in profiles/).
TRAFFIC_RATIO = {
    "orth_b6": (0.9972, "ncu dram bytes of gm_dc_dot + gm_dc_update at Arnoldi step j = 99 with the 6-byte basis "
                        "(412.2 MB) over the bytes they move (413.3 MB), profiles/gm_dc_arnoldi__advdiff_s2048_N64.md"),
}


def kernel_rows(st, step_ms, hbm, dcgs=False):
    rows = {}
    if st.gemm_launches:
        a = st.gemm_flops / (st.gemm_ms * 1e-3) / 1e12
        rows["gemm_fp64"] = {"kernel": "gemm_streamk_kernel<double> (FP64 covariance / factor products)",
                             "bound": "alu", "achieved": a, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "frac": a / FP64_PEAK_TFLOPS, "launches": st.gemm_launches,
                             "ms_per_launch": st.gemm_ms / st.gemm_launches,
                             "flops_per_launch": st.gemm_flops / st.gemm_launches,
                             "share_of_step": st.gemm_ms / step_ms,
                             "peak_source": "derived: 152 SM x 4 FP64 flop/clk x 2.07 GHz"}
    if st.gemmdf_launches:
        a = st.gemmdf_flops / (st.gemmdf_ms * 1e-3) / 1e12
        rows["gemm_df32"] = {"kernel": "gemm_streamk_df32_kernel (double-float covariance / factor products)",
                             "bound": "alu", "achieved": a, "peak": DF32_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "frac": a / DF32_PEAK_TFLOPS, "launches": st.gemmdf_launches,
                             "ms_per_launch": st.gemmdf_ms / st.gemmdf_launches,
                             "flops_per_launch": st.gemmdf_flops / st.gemmdf_launches,
                             "share_of_step": st.gemmdf_ms / step_ms,
                             "peak_source": "derived: FP32 pipe (152 SM x 128 lanes x 2.07 GHz) / 12 "
                                            "FP32 lane operations per double-float multiply-add"}
    if st.gemmtc_launches:
        ms1 = st.gemmtc_ms / st.gemmtc_launches
        # the byte floor of the per-unit accounting: each FP64 operator entry read once, vectors once;
        # the digit form (what the kernel moves: 14 B per operator entry) is reported beside it
        a_hbm = st.gemmtc_alg_bytes / (st.gemmtc_ms * 1e-3) / 1e9
        a_dig = st.gemmtc_bytes / (st.gemmtc_ms * 1e-3) / 1e9
        a_tc = st.gemmtc_mma_flops / (st.gemmtc_ms * 1e-3) / 1e12
        bf16 = peaks().get("bf16_tflops")
        f_hbm = (a_hbm / hbm) if hbm else None
        f_tc = (a_tc / bf16) if bf16 else None
        tensor_bound = f_tc is not None and (f_hbm is None or f_tc >= f_hbm)
        rows["gemm_tc"] = {"kernel": "gemm_tc_kernel (Ozaki digit products on tcgen05; one-column products "
                                     "in double-float)",
                           "bound": "tensor" if tensor_bound else "hbm",
                           "achieved": a_tc if tensor_bound else a_hbm,
                           "peak": bf16 if tensor_bound else hbm,
                           "unit": "TFLOP/s" if tensor_bound else "GB/s",
                           "frac": f_tc if tensor_bound else f_hbm,
                           "hbm": {"achieved_gbs": a_hbm, "frac": f_hbm,
                                   "bytes": "FP64 operator entries (their triangle) once, vectors once"},
                           "digit_form": {"achieved_gbs": a_dig, "frac": (a_dig / hbm) if hbm else None,
                                          "bytes_per_launch": st.gemmtc_bytes / st.gemmtc_launches,
                                          "bytes": "digit tiles (14 B per operator entry), GEMV operands, "
                                                   "vector digits, partial tiles: what the kernel moves"},
                           "tensor": {"achieved_tflops_bf16": a_tc, "frac": f_tc},
                           "fp64_class_tflops": st.gemmtc_flops / (st.gemmtc_ms * 1e-3) / 1e12,
                           "launches": st.gemmtc_launches, "ms_per_launch": ms1,
                           "flops_per_launch": st.gemmtc_flops / st.gemmtc_launches,
                           "bytes_per_launch": st.gemmtc_alg_bytes / st.gemmtc_launches,
                           "mma_flops_per_launch": st.gemmtc_mma_flops / st.gemmtc_launches,
                           "share_of_step": st.gemmtc_ms / step_ms,
                           "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst) / hbm_gbs (measured)"}
    if st.gemm32_launches:
        a = st.gemm32_flops / (st.gemm32_ms * 1e-3) / 1e12
        rows["gemm_fp32"] = {"kernel": "gemm_streamk_kernel<float> (FP32 inner-solve products)",
                             "bound": "alu", "achieved": a, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "frac": a / FP32_PEAK_TFLOPS, "launches": st.gemm32_launches,
                             "ms_per_launch": st.gemm32_ms / st.gemm32_launches,
                             "flops_per_launch": st.gemm32_flops / st.gemm32_launches,
                             "share_of_step": st.gemm32_ms / step_ms,
                             "peak_source": "derived: 152 SM x 256 FP32 flop/clk x 2.07 GHz"}
    if st.circ_launches:
        a = st.circ_flops / (st.circ_ms * 1e-3) / 1e12
        rows["circ_fft"] = {"kernel": "circ_kernel / band_kernel (circulant B, Q: FP64 FFT in 8-CTA clusters, "
                                      "or the banded taps)",
                            "bound": "alu", "achieved": a, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                            "frac": a / FP64_PEAK_TFLOPS, "launches": st.circ_launches,
                            "ms_per_launch": st.circ_ms / st.circ_launches,
                            "flops_per_launch": st.circ_flops / st.circ_launches,
                            "bytes_per_launch": st.circ_bytes / st.circ_launches,
                            "hbm_gbs": st.circ_bytes / (st.circ_ms * 1e-3) / 1e9,
                            "share_of_step": st.circ_ms / step_ms,
                            "peak_source": "derived: 152 SM x 4 FP64 flop/clk x 2.07 GHz; flops counted as "
                                           "5 s log2 s per complex transform, 2 per band tap"}
    if st.pt_launches:
        a = st.pt_bytes / (st.pt_ms * 1e-3) / 1e9
        rows["pertime"] = {"kernel": "pertime_kernel (per-time R_i family products)", "bound": "hbm",
                           "achieved": a, "peak": hbm, "unit": "GB/s", "frac": (a / hbm) if hbm else None,
                           "launches": st.pt_launches, "ms_per_launch": st.pt_ms / st.pt_launches,
                           "bytes_per_launch": st.pt_bytes / st.pt_launches, "share_of_step": st.pt_ms / step_ms,
                           "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}
    if st.orth_launches:
        a = st.orth_bytes / (st.orth_ms * 1e-3) / 1e9
        name = ("gm_dc_dot/gm_dc_update (delayed-CGS2 Arnoldi passes)" if dcgs
                else "gm_mdot/gm_mupdate (Arnoldi CGS2 passes)")
        rows["orth"] = {"kernel": name, "bound": "hbm", "achieved": a,
                        "peak": hbm, "unit": "GB/s", "frac": (a / hbm) if hbm else None,
                        "launches": st.orth_launches, "ms_per_launch": st.orth_ms / st.orth_launches,
                        "bytes_per_launch": st.orth_bytes / st.orth_launches, "share_of_step": st.orth_ms / step_ms,
                        "bytes": "FP64-equivalent: 8 B per basis entry read or written, w and v at 8 B",
                        "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}
        if st.orth_moved_bytes and abs(st.orth_moved_bytes - st.orth_bytes) > 1e-6 * st.orth_bytes:
            m = st.orth_moved_bytes / (st.orth_ms * 1e-3) / 1e9
            rows["orth"]["moved"] = {"achieved_gbs": m, "frac": (m / hbm) if hbm else None,
                                     "bytes_per_launch": st.orth_moved_bytes / st.orth_launches,
                                     "bytes": "what the passes move: 6 B per basis entry (FP32 + BF16)"}
    return rows


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2105_06975_gb300 import wc4d, workload as W

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    from paper_2105_06975_gb300.ranks import window_seed
    w = W.SCALE
    seed = window_seed(args.seed, rank)
    dr = W.draws(w, seed)
    ce = args.check_every
    modes = {
        "fp64": wc4d.make_opts(precond=args.precond, k=args.k, rhat=args.rhat, tol=1e-6, maxit=args.maxit,
                               check_every=ce),
        "df32": wc4d.make_opts(precond=args.precond, k=args.k, rhat=args.rhat, tol=1e-6, maxit=args.maxit,
                               precision="df32", check_every=ce),
        "ozaki": wc4d.make_opts(precond=args.precond, k=args.k, rhat=args.rhat, tol=1e-6, maxit=args.maxit,
                                precision="ozaki", check_every=ce),
    }
    # Rhat^-1 as one product with the explicit inverse (one dependency level less per preconditioner apply)
    if args.chosen == "ozaki_rinv" or (args.modes and "ozaki_rinv" in args.modes.split(",")):
        modes["ozaki_rinv"] = wc4d.make_opts(precond=args.precond, k=args.k, rhat=args.rhat, tol=1e-6,
                                             maxit=args.maxit, precision="ozaki", check_every=ce, rinv_explicit=True)
    # the same with the 6-byte Arnoldi basis (a quarter fewer bytes in both basis passes)
    if args.chosen == "ozaki_rinv_b6" or (args.modes and "ozaki_rinv_b6" in args.modes.split(",")):
        modes["ozaki_rinv_b6"] = wc4d.make_opts(precond=args.precond, k=args.k, rhat=args.rhat, tol=1e-6,
                                                maxit=args.maxit, precision="ozaki", check_every=ce,
                                                rinv_explicit=True, basis_bytes=6)
    # the same reading B's s x s entries for its one-column products (its first row otherwise: B is Toeplitz)
    if args.modes and "ozaki_rinv_b6_dense" in args.modes.split(","):
        modes["ozaki_rinv_b6_dense"] = wc4d.make_opts(precond=args.precond, k=args.k, rhat=args.rhat, tol=1e-6,
                                                      maxit=args.maxit, precision="ozaki", check_every=ce,
                                                      rinv_explicit=True, basis_bytes=6,
                                                      toeplitz_gemv=wc4d.WC4D_TOEPLITZ_OFF)
    if args.chosen == "ozaki_fft_rinv_b6" or (args.modes and "ozaki_fft_rinv_b6" in args.modes.split(",")):
        modes["ozaki_fft_rinv_b6"] = wc4d.make_opts(precond=args.precond, k=args.k, rhat=args.rhat, tol=1e-6,
                                                    maxit=args.maxit, precision="ozaki", check_every=ce,
                                                    covprod="fft", rinv_explicit=True, basis_bytes=6)
    # circulant B and Q applied by FFT (Sec. 6.1), the R family as in the base mode
    for m in ("fp64", "df32", "ozaki"):
        if args.chosen == m + "_fft" or (args.modes and m + "_fft" in args.modes.split(",")):
            modes[m + "_fft"] = wc4d.make_opts(precond=args.precond, k=args.k, rhat=args.rhat, tol=1e-6,
                                               maxit=args.maxit, precision=m, check_every=ce, covprod="fft")
    if args.chosen == "df32p32" or (args.modes and "df32p32" in args.modes.split(",")):
        # FP32 preconditioner: only for covariances with kappa * eps32 << 1 (not this workload's R)
        modes["df32p32"] = wc4d.make_opts(precond=args.precond, k=args.k, rhat=args.rhat, tol=1e-6,
                                          maxit=args.maxit, precision="df32p32")
    if args.mixed or args.chosen == "mixed":
        modes["mixed"] = wc4d.make_opts(precond=args.precond, k=args.k, rhat=args.rhat, tol=1e-6,
                                        maxit=min(args.maxit, 200), precision="mixed", inner_iters=args.inner)
    if args.modes:
        keep = args.modes.split(",")
        modes = {m: o for m, o in modes.items() if m in keep}
    G = wc4d.Problem.from_workload(w, dr, wc4d.make_opts(precond=args.precond, k=args.k, rhat=args.rhat),
                                   stream=stream.cuda_stream)
    rhs = G.synthesize_rhs(dr)
    G.close()
    x = torch.zeros(w.n, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    hbm = peaks().get("hbm_gbs")

    split = []   # host-side (setup ms, solve ms) per step: setup synchronises, so this is a clean cut

    def step(opts):
        t0 = time.perf_counter()
        G = wc4d.Problem.from_workload(w, dr, opts, stream=stream.cuda_stream)
        t1 = time.perf_counter()
        _, info = G.solve(rhs, x)
        t2 = time.perf_counter()
        G.close()
        split.append(((t1 - t0) * 1e3, (t2 - t1) * 1e3))
        return info

    results = {}
    clk = ClockSampler(local)
    if not args.no_clocks:
        clk.start()
    def timed(opts, profiled):
        """K steps between barriers and device syncs, each bracketed by CUDA
        events on the launching stream; L2 flushed before every step."""
        if profiled:
            wc4d.wc4d_reset_stats()
            wc4d.wc4d_set_profiling(True)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ev, infos = [], []
        split.clear()
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos.append(step(opts))
            e1.record(stream)
            ev.append((e0, e1))
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        st = None
        if profiled:
            wc4d.wc4d_set_profiling(False)
            st = wc4d.wc4d_get_stats()
        return sum(a.elapsed_time(b) for a, b in ev), infos, st

    for mode, opts in modes.items():
        for _ in range(args.warmup):
            step(opts)
        # the headline steps run without the library's per-launch profiling
        # events; a second, profiled pass of the same K steps gives the
        # per-kernel rows (time per launch, algorithmic work)
        step_ms, infos, _ = timed(opts, False)
        split_plain = list(split)
        prof_ms, _, st = timed(opts, True)
        split[:] = split_plain
        ms = step_ms / args.steps
        if world > 1:
            tt = torch.tensor([ms], device=dev)
            torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
            ms = float(tt.item())
        assert all(i.status == 0 for i in infos), [i.as_dict() for i in infos]
        results[mode] = {"ms": ms, "value": world * 1e3 / ms, "infos": infos, "stats": st,
                         "kernels": kernel_rows(st, prof_ms, hbm, dcgs=mode in ("df32", "df32p32", "ozaki", "df32_fft",
                                                                              "ozaki_fft", "ozaki_rinv", "ozaki_rinv_b6",
                                                                              "ozaki_fft_rinv_b6")),
                         "profiled_ms_per_step": prof_ms / args.steps,
                         "setup_ms": statistics.mean(a for a, _ in split),
                         "solve_ms": statistics.mean(b for _, b in split)}
    # the paper's other preconditioner and the circulant products on the same window (Sec. 2.2, 6.1):
    # P_D + MINRES and P_I + GMRES with B, Q by FFT, timed like the headline steps
    comparisons = {}
    if not args.no_comparisons and world == 1:
        for name, o in (("PD_minres_ozaki_fft", wc4d.make_opts(precond="PD", k=args.k, rhat=args.rhat, tol=1e-6,
                                                               maxit=3000, precision="ozaki", covprod="fft",
                                                               check_every=ce)),
                        ("PI_gmres_ozaki_fft", wc4d.make_opts(precond="PI", k=args.k, rhat=args.rhat, tol=1e-6,
                                                              maxit=args.maxit, precision="ozaki", covprod="fft",
                                                              check_every=ce)),
                        ("PD_minres_ozaki", wc4d.make_opts(precond="PD", k=args.k, rhat=args.rhat, tol=1e-6,
                                                           maxit=3000, precision="ozaki", check_every=ce)),
                        # the chosen mode with reduced-precision preconditioner products: 5 of the 7 BF16
                        # digits (about 34-bit operands) in P_I's tensor-core products, the flexible GMRES
                        # keeping the computed P^-1 u (A v and the residual stay FP64-class)
                        ("PI_gmres_ozaki_rinv_b6_prec5", wc4d.make_opts(precond="PI", k=args.k, rhat=args.rhat,
                                                                        tol=1e-6, maxit=args.maxit, precision="ozaki",
                                                                        check_every=ce, rinv_explicit=True,
                                                                        basis_bytes=6, prec_digits=5))):
            if name == "PI_gmres_ozaki_fft" and args.precond == "PI" and "ozaki_fft" in results:
                continue
            for _ in range(max(1, args.warmup // 2)):
                step(o)
            c_ms, c_infos, _ = timed(o, False)
            if not all(i.status == 0 for i in c_infos):  # reported, not fatal: a comparison, not the headline
                comparisons[name] = {"converged": False, "status": [i.status for i in c_infos],
                                     "iterations": statistics.mean(i.iters for i in c_infos),
                                     "relres_true_max": max(i.relres_true for i in c_infos)}
                continue
            comparisons[name] = {"solves_per_s": 1e3 * args.steps / c_ms, "ms_per_step": c_ms / args.steps,
                                 "iterations": statistics.mean(i.iters for i in c_infos),
                                 "relres_true_max": max(i.relres_true for i in c_infos),
                                 "setup_ms_host": statistics.mean(a for a, _ in split),
                                 "solve_ms_host": statistics.mean(b for _, b in split)}
    clocks = clk.stop()
    chosen = results[args.chosen] if args.chosen in results else next(iter(results.values()))
    fp64 = results.get("fp64", chosen)
    iters = [i.iters for i in chosen["infos"]]
    inner = [i.inner_iters for i in chosen["infos"]]

    # end to end through the C ABI with host buffers: H2D of the observation
    # indices and the right-hand side, D2H of the solution, inside the timing
    rhs_h = rhs.cpu().numpy()
    x_h = np.zeros_like(rhs_h)
    obs_h = np.ascontiguousarray(dr.obs_idx, dtype=np.int32)
    e2e_t = []
    for i in range(0 if args.no_e2e else max(2, args.steps // 2) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Gh = wc4d.Problem(w.s, w.N, w.p, obs_h, modes[args.chosen], stencil=w.stencil(), soar_b=w.soar_b,
                          soar_q=w.soar_q, soar_r=w.soar_r, stream=stream.cuda_stream)
        _, info = Gh.solve(rhs_h, x_h)
        Gh.close()
        if i > 0:
            e2e_t.append(time.perf_counter() - t0)
        assert info.status == 0
    e2e_val = world / statistics.mean(e2e_t) if e2e_t else None

    ks = chosen["kernels"]
    dom = max(ks.values(), key=lambda r: r["share_of_step"]) if ks else None
    roof = None
    if dom is not None:
        roof = {k: dom[k] for k in ("kernel", "bound", "achieved", "peak", "unit", "frac", "peak_source",
                                    "share_of_step")}
        roof["traffic"] = GEMM_DF32_TRAFFIC_BYTES if dom["kernel"].startswith("gemm_streamk_df32") else None
        if roof["traffic"] is not None:
            roof["traffic_source"] = ("ncu dram bytes read+write per launch, mean of one GMRES step's three "
                                      "product launches (profiles/gemm_streamk_df32__advdiff_s2048_N64.md)")
        dom_key = next(k for k, r in ks.items() if r is dom)
        # the 6-byte basis passes have their own capture, scaled by the bytes they move
        tkey = dom_key + "_b6" if "moved" in dom else dom_key
        if tkey in TRAFFIC_RATIO and dom.get("bytes_per_launch"):
            ratio, src = TRAFFIC_RATIO[tkey]
            base = dom["moved"]["bytes_per_launch"] if "moved" in dom else dom["bytes_per_launch"]
            roof["traffic"] = ratio * base
            roof["traffic_source"] = src + ("; scaled to this run's mean bytes moved per launch" if "moved" in dom
                                            else "; scaled to this run's mean algorithmic bytes per launch")
    # whole-solve bound: the FP64-class products at the DF32 peak vs the Arnoldi and operator bytes at HBM
    st_c = chosen["stats"]
    solve_roof = None
    bf16 = peaks().get("bf16_tflops")
    if st_c.gemmtc_launches and hbm and bf16:
        # tensor-core mode: digit products at the BF16 peak vs the Arnoldi, digit-tile and GEMV bytes at HBM
        steps_n = max(args.steps, 1)
        t_tc = st_c.gemmtc_mma_flops / steps_n / (bf16 * 1e12) * 1e3
        t_hbm = (st_c.orth_bytes + st_c.gemmtc_bytes) / steps_n / (hbm * 1e9) * 1e3
        t_roof = max(t_tc, t_hbm)
        solve_roof = {"bound": "tensor" if t_tc >= t_hbm else "hbm", "t_tensor_ms": t_tc, "t_hbm_ms": t_hbm,
                      "t_roof_ms": t_roof, "ms_per_step": chosen["ms"], "frac": t_roof / chosen["ms"],
                      "note": "lower bound of one step from the digit-product FLOPs (measured BF16 peak) and the "
                              "Arnoldi + operator-digit + GEMV bytes (measured HBM); setup and small kernels "
                              "count as time only"}
    elif st_c.gemmdf_launches and hbm:
        steps_n = max(args.steps, 1)
        t_alu = st_c.gemmdf_flops / steps_n / (DF32_PEAK_TFLOPS * 1e12) * 1e3
        t_hbm = (st_c.orth_bytes + st_c.gemmdf_launches * GEMM_DF32_TRAFFIC_BYTES) / steps_n / (hbm * 1e9) * 1e3
        t_roof = max(t_alu, t_hbm)
        solve_roof = {"bound": "alu" if t_alu >= t_hbm else "hbm", "t_alu_ms": t_alu, "t_hbm_ms": t_hbm,
                      "t_roof_ms": t_roof, "ms_per_step": chosen["ms"], "frac": t_roof / chosen["ms"],
                      "note": "lower bound of one step from the product FLOPs (DF32 peak) and the Arnoldi + "
                              "operator bytes (measured HBM); setup and small kernels count as time only"}
    line = {
        "metric": METRIC, "value": chosen["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": chosen["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": MODE_DTYPE[args.chosen], "data": "synthetic", "impl": "gpu",
        "config": {**workload_config(args, w), "mode": MODE_DESC[args.chosen].format(inner=args.inner, pc=args.precond),
                   "parallelism": f"windows x{world}"},
        "iterations": {"mean": statistics.mean(iters), "inner_total_mean": statistics.mean(inner)},
        "modes": {m: {"solves_per_s": r["value"], "ms_per_step": r["ms"],
                      "iterations": statistics.mean(i.iters for i in r["infos"]),
                      "setup_ms_host": r["setup_ms"], "solve_ms_host": r["solve_ms"]} for m, r in results.items()},
        "relres_true_max": max(i.relres_true for i in chosen["infos"]),
        "comparisons": comparisons,
        "fp64_solves_per_s": fp64["value"],
        "chosen_over_fp64": chosen["value"] / fp64["value"],
        "roofline": roof,
        "roofline_step": solve_roof,
        "kernels": ks,
        "kernels_fp64_mode": fp64["kernels"],
        "gpu_launches": int(chosen["stats"].launches),
        "gpu_launches_fp64_mode": int(fp64["stats"].launches),
        "clocks": clocks,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(w.n * 8 + w.p * 4),
                "d2h_bytes_per_step": int(w.n * 8)},
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_solve(args, w, dr)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def build_batch(args, wc4d, W, opts):
    """Set up the batched workload's windows on the device (no oracle): SOAR
    covariances built by the library; advection-diffusion right-hand sides
    synthesised on the device; Lorenz-96 windows linearised about their device
    background forecast, with observations = forecast + sqrt(sigma_o^2) z."""
    import numpy as np
    from paper_2105_06975_gb300.ranks import dist_info as _di, partition_by_cost
    rank, world, _ = _di()
    wins = W.batch_windows(args.batch, args.seed)
    mine = partition_by_cost([(w.s * w.s + w.p * w.p) * (w.N + 1) for w, _ in wins], world)[rank]
    probs, rhs, meta = [], [], []
    for w, seed in (wins[i] for i in mine):
        dr = W.draws(w, seed)
        if w.model == "advdiff":
            G = wc4d.Problem.from_workload(w, dr, opts)
            r = G.synthesize_rhs(dr)
        else:
            spo = w.steps_per_obs
            G = wc4d.Problem(w.s, w.N, w.p, dr.obs_idx, opts, banded=True, band_lo=8 * spo, band_hi=4 * spo,
                             soar_b=w.soar_b, soar_q=w.soar_q, soar_r=w.soar_r)
            xb = w.forcing + dr.x0_pert
            y0 = np.zeros((w.N + 1, w.p))
            traj, _, _ = G.l96_gauss_newton(w.forcing, w.dt, spo, 0, xb, y0)
            y = traj[:, dr.obs_idx] + np.sqrt(w.soar_r[0]) * dr.z_r
            import torch
            r = torch.from_numpy(G.l96_linearize(w.forcing, w.dt, spo, xb, y, traj)).cuda()
        probs.append(G)
        rhs.append(r)
        meta.append((w.model, w.s, w.N, w.p))
    return probs, rhs, meta


def run_batch(args):
    import numpy as np
    import torch

    from paper_2105_06975_gb300 import wc4d, workload as W

    from paper_2105_06975_gb300.ranks import job_throughput, sum_over_ranks
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl")
    opts = wc4d.make_opts(precond=args.precond, k=args.k, rhat=args.rhat, tol=1e-6, maxit=args.batch_maxit,
                          precision=args.precision, check_every=args.check_every, rinv_explicit=args.rinv)
    t0 = time.perf_counter()
    probs, rhs, meta = build_batch(args, wc4d, W, opts)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    xs = [torch.zeros_like(r) for r in rhs]
    for _ in range(args.warmup):
        _, infos, code = wc4d.solve_batch(probs, rhs, xs, workers=args.workers)
    clk = ClockSampler(local)
    if not args.no_clocks:
        clk.start()
    wc4d.wc4d_reset_stats()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t1 = time.perf_counter()
    codes, all_infos = [], []
    for _ in range(args.steps):
        _, infos, code = wc4d.solve_batch(probs, rhs, xs, workers=args.workers)
        codes.append(code)
        all_infos.append(infos)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - t1
    clocks = clk.stop()
    st = wc4d.wc4d_get_stats()
    dev = torch.device("cuda", local)
    value, ms = job_throughput(len(probs), wall * 1e3 / args.steps, device=dev if world > 1 else None)
    infos = all_infos[-1]
    its = [i.iters for i in infos]
    ok = int(sum_over_ranks(sum(i.status == 0 for i in infos), device=dev if world > 1 else None))
    if rank != 0:
        for G in probs:
            G.close()
        return
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "df32 products (2 x f32, ~48-bit) / f64 recurrences", "data": "synthetic",
           "impl": "gpu",
           "config": {"workload": f"{args.batch} independent windows, s=4U{{32..512}}, N=U{{8..96}}, p=s/2|s/4, "
                                  "advection-diffusion | Lorenz-96 (dt 1e-4), SOAR covariances",
                      "precond": args.precond, "lhat": f"L_M({args.k})", "rhat": args.rhat, "tol": 1e-6,
                      "maxit_per_window": args.batch_maxit, "workers": args.workers,
                      "check_every": args.check_every,
                      "step": "wc4d_solve_batch over all windows (set up once, outside the timed region)",
                      "l2": "inputs larger than L2 (the windows' operators total tens of GB)"},
           "windows_converged": ok, "windows_per_rank_rank0": len(probs),
           "iterations": {"mean": float(np.mean(its)), "max": int(max(its))},
           "relres_true_max": max(i.relres_true for i in infos), "setup_s": setup_s,
           "gpu_launches": st.launches // max(args.steps, 1), "clocks": clocks,
           "timing": "host wall clock around the blocking batch call, device synchronised on both sides",
           "statuses": sorted(set(codes))}
    print(json.dumps(out))
    for G in probs:
        G.close()


def run_learned(args):
    """Learned Schur block (trained on the device, outside the timed region)
    against the plain block-diagonal preconditioner: advection-diffusion
    s=1024, N=32, p=512, P_D with L_M(k), solves to true relres 1e-6."""
    import numpy as np
    import torch

    from paper_2105_06975_gb300 import wc4d, workload as W

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    w = W.SCALE.with_(name="learned-advdiff", s=1024, N=32, p=512)
    dr = W.draws(w, args.seed * 1000 + rank)
    k = min(args.k, w.N + 1)
    arms = {
        "learned_gmres": wc4d.make_opts(precond="PD", k=k, shat="learned", krylov="gmres", tol=1e-6,
                                        maxit=args.maxit, precision=args.precision),
        "plain_gmres": wc4d.make_opts(precond="PD", k=k, krylov="gmres", tol=1e-6, maxit=args.maxit,
                                      precision=args.precision),
        "plain_minres": wc4d.make_opts(precond="PD", k=k, krylov="minres", tol=1e-6, maxit=20000,
                                       precision=args.precision),
    }
    probs = {a: wc4d.Problem.from_workload(w, dr, o) for a, o in arms.items()}
    rhs = probs["plain_gmres"].synthesize_rhs(dr)
    t0 = time.perf_counter()
    rep = probs["learned_gmres"].precond_train(pairs=args.pairs, hidden=32, batch=64, epochs=args.epochs,
                                               lr=1e-3, seed=args.seed + 1, loss=args.loss)
    train_s = time.perf_counter() - t0
    out_arms = {}
    for a, G in probs.items():
        x = torch.zeros_like(rhs)
        for _ in range(args.warmup):
            G.solve(rhs, x)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = [G.solve(rhs, x)[1] for _ in range(args.steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        out_arms[a] = {"solves_per_s": 1e3 / ms, "ms_per_solve": ms, "iterations": infos[-1].iters,
                       "status": infos[-1].status, "relres_true": infos[-1].relres_true,
                       "precond_fallback": infos[-1].precond_fallback}
    best = out_arms["learned_gmres"]
    line = {"metric": METRIC, "value": best["solves_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": best["ms_per_solve"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "df32 products / f64 recurrences; learned block FP32", "data": "synthetic",
            "impl": "gpu",
            "config": {"workload": f"advection-diffusion window s={w.s} N={w.N} p={w.p} (n={w.n}), SOAR B/Q/R; "
                                   "learned Schur block in GMRES vs plain P_D",
                       "precond": "PD", "lhat": f"L_M({k})", "tol": 1e-6, "pairs": args.pairs,
                       "epochs": args.epochs, "hidden": 32, "loss": args.loss,
                       "step": "one solve with the problem set up and the net trained (outside the timed region)",
                       "l2": "operators (3 x 8 MB B/Q/R plus factors) and the n-vectors exceed L2 only in part"},
            "arms": out_arms, "training": {k_: (round(v, 5) if isinstance(v, float) else v)
                                           for k_, v in rep.as_dict().items()},
            "train_wall_s": train_s}
    print(json.dumps(line))
    for G in probs.values():
        G.close()


def run_heat(args):
    """The heat-equation window of Sec. 7.2 at its largest size: s = 50,000,
    N = 5, p = 12,500 random observed points, B and Q the banded circulant
    modified SOAR of Sec. 6.1 (applied through their taps), R the chordal SOAR
    over the observed points, P_I + GMRES with L_M(k), right-hand side
    (0, z_r, 0).  A step is the device problem build (Rhat = R factor and
    inverse, p = 12,500) and the solve to true relres 1e-6."""
    import torch

    from paper_2105_06975_gb300 import wc4d, workload as W
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    w = W.HEAT_SOAR_R
    dr = W.draws(w, args.seed * 1000 + rank)
    bands = w.heat_bands()
    rhs = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    rhs[w.s * (w.N + 1):w.s * (w.N + 1) + w.p * (w.N + 1)] = torch.from_numpy(dr.z_r.ravel())
    x = torch.zeros_like(rhs)
    precision = args.precision
    opts = wc4d.make_opts(precond="PI", k=args.k, tol=1e-6, maxit=args.maxit, precision=precision,
                          check_every=args.check_every)
    stream = torch.cuda.current_stream()

    def step():
        G = wc4d.Problem(w.s, w.N, w.p, dr.obs_idx, opts, bands=bands, band_lo=1, band_hi=1,
                         msoar=(w.msoar_b, w.msoar_q, dr.extra["psi"]), soar_r=w.soar_r,
                         stream=stream.cuda_stream)
        _, info = G.solve(rhs, x)
        G.close()
        return info
    for _ in range(args.warmup):
        step()
    clk = ClockSampler(local)
    if not args.no_clocks:
        clk.start()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = [step() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    clocks = clk.stop()
    wc4d.wc4d_reset_stats()
    wc4d.wc4d_set_profiling(True)
    torch.cuda.synchronize()
    p0 = time.perf_counter()
    step()
    torch.cuda.synchronize()
    prof_ms = (time.perf_counter() - p0) * 1e3
    wc4d.wc4d_set_profiling(False)
    st = wc4d.wc4d_get_stats()
    hbm = peaks().get("hbm_gbs")
    ks = kernel_rows(st, prof_ms, hbm, dcgs=precision in ("df32", "ozaki"))
    dom = max(ks.values(), key=lambda r: r["share_of_step"]) if ks else None
    roof = ({k: dom[k] for k in ("kernel", "bound", "achieved", "peak", "unit", "frac", "peak_source",
                                 "share_of_step")} if dom else None)
    if roof:
        roof["traffic"] = None
    assert all(i.status == 0 for i in infos), [i.as_dict() for i in infos]
    line = {"metric": METRIC, "value": 1e3 / ms, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": MODE_DTYPE.get(precision, precision), "data": "synthetic", "impl": "gpu",
            "config": {"workload": f"heat equation (Sec. 7.2) s={w.s} N={w.N} p={w.p} (n={w.n}); banded "
                                   "circulant modified SOAR B, Q; SOAR R over the observed points",
                       "precond": "PI", "lhat": f"L_M({args.k})", "rhat": "exact", "krylov": "GMRES (no restart)",
                       "tol": 1e-6, "step": "device problem build (Rhat factor and inverse, p = 12,500) + solve",
                       "l2": "inputs larger than L2 (each R-family operator 1.25 GB)"},
            "iterations": statistics.mean(i.iters for i in infos),
            "relres_true_max": max(i.relres_true for i in infos),
            "solve_ms_mean": statistics.mean(i.ms for i in infos),
            "roofline": roof, "kernels": ks, "gpu_launches": int(st.launches), "clocks": clocks}
    print(json.dumps(line), flush=True)


def run_profile(args):
    """The hot kernels at the scale workload's sizes, for ncu captures: 4 x
    (A v, P_I^-1 v) through the C ABI, then one GMRES solve capped at --maxit
    steps (tolerance unreachable, so the Arnoldi passes run up to j = maxit-1).
    About 1 GB on the device at --maxit 110.  Prints one JSON line of CUDA-event
    timings (not a benchmark line)."""
    import torch

    from paper_2105_06975_gb300 import wc4d, workload as W
    torch.cuda.set_device(0)
    w = W.SCALE
    dr = W.draws(w, args.seed)
    base = args.chosen.replace("_fft", "").replace("_rinv", "").replace("_b6", "")
    # the 6-byte basis refuses tolerances below 1e-7; the scale window needs about 150 steps to reach it,
    # so a --maxit up to about 140 still runs every step
    o = wc4d.make_opts(precond=args.precond, k=args.k, rhat=args.rhat,
                       tol=1e-7 if args.chosen.endswith("_b6") else 1e-30, maxit=args.maxit,
                       precision=base if base in ("fp64", "df32", "ozaki") else "ozaki",
                       covprod="fft" if "_fft" in args.chosen else "dense",
                       krylov="gmres" if args.precond == "PI" else "minres",
                       rinv_explicit=("_rinv" in args.chosen), basis_bytes=6 if args.chosen.endswith("_b6") else 0)
    G = wc4d.Problem.from_workload(w, dr, o)
    v = torch.from_numpy(W.random_vector(w.n, 3)).cuda()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for _ in range(4):
        G.apply_saddle(v)
        G.apply_precond(args.precond, v)
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(4):
        G.apply_saddle(v)
    ev[1].record()
    for _ in range(4):
        G.apply_precond(args.precond, v)
    ev[2].record()
    torch.cuda.synchronize()
    # the library's own accounting of one A v launch and one P^-1 v (two launches)
    acct = {}
    for name, fn in (("apply_saddle", lambda: G.apply_saddle(v)), ("apply_precond", lambda: G.apply_precond(args.precond, v))):
        wc4d.wc4d_set_profiling(1)
        wc4d.wc4d_reset_stats()
        fn()
        st = wc4d.wc4d_get_stats()
        wc4d.wc4d_set_profiling(0)
        acct[name] = {"product_launches": st.gemmtc_launches + st.gemmdf_launches,
                      "bytes": st.gemmtc_bytes, "fp64_class_flops": st.gemmtc_flops + st.gemmdf_flops,
                      "bf16_mma_flops": st.gemmtc_mma_flops, "ms": st.gemmtc_ms + st.gemmdf_ms}
    rhs = G.synthesize_rhs(dr)
    x = torch.zeros_like(rhs)
    t0 = time.perf_counter()
    wc4d.wc4d_solve(G.h, rhs.data_ptr(), x.data_ptr(), False, wc4d.WC4D_MEM_DEVICE, raise_on_error=False)
    torch.cuda.synchronize()
    G.close()
    print(json.dumps({"workload": "profile", "precision": o.precision, "apply_saddle_ms": ev[0].elapsed_time(ev[1]) / 4,
                      "apply_precond_ms": ev[1].elapsed_time(ev[2]) / 4, "product_accounting": acct,
                      "solve_steps": args.maxit, "solve_ms": (time.perf_counter() - t0) * 1e3}))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "profile":
        run_profile(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "heat":
        run_heat(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
