/*
 * wc4d -- weak-constraint 4D-Var saddle-point solver, C ABI.
 *
 * Tabeart & Pearson, "Saddle point preconditioners for weak-constraint
 * 4D-Var".  The library solves the inner-loop saddle-point system
 * (Sec. 2.1, Eq. saddlepointsystem)
 *
 *     [ D   0   L ] [d_eta]   [b]
 *     [ 0   R   H ] [d_nu ] = [d]          A = Eq. saddlepointA
 *     [ L^T H^T 0 ] [d_x  ]   [0]
 *
 * with D = blkdiag(B, Q_1..Q_N), R = blkdiag(R_0..R_N), H = blkdiag(H_i),
 * L block lower bidiagonal with I on the diagonal and -M_i below it
 * (Eq. def:L), preconditioned by the block-diagonal P_D or the inexact
 * constraint P_I (Eq. prec) built from Lhat = L_M(k) (Definition 1) and a
 * reconditioned Rhat (Sec. 5, Alg. 1 and 2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Vectors of length n = (2s+p)(N+1) are time-major FP64:
 *       [eta_0..eta_N (each s) | nu_0..nu_N (each p) | x_0..x_N (each s)],
 *   each block contiguous, so block k of a part is the column k of an
 *   s x (N+1) (or p x (N+1)) column-major matrix.
 * - Q_i = Q for every time level.  By default R_i = R and H_i selects the
 *   same sorted observed grid points at every time (Sec. 6.1); with
 *   wc4d_problem_desc.p_t every time level has its own set and R_i.
 * - Dense matrices are column-major, symmetric, FP64.
 * - "device" pointers are CUDA global-memory addresses on the current
 *   device (e.g. torch tensor data_ptr()); "host" pointers are ordinary CPU
 *   memory.  The library never takes ownership of caller memory; everything
 *   it needs is copied into library-owned device buffers at setup.
 * - All work is ordered on the CUDA stream given at setup.  Calls return
 *   after the work is enqueued, except where stated (solve: returns after
 *   the solution is final, because the convergence test reads a device flag).
 * - Every call returns a status code (WC4D_OK = 0 on success).  No C++
 *   exception crosses the ABI.  The message of the last failure on the
 *   calling thread is returned by wc4d_last_error().
 * - A problem handle must not be used from two host threads at once.
 */
#ifndef WC4D_H
#define WC4D_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
enum {
  WC4D_OK = 0,
  WC4D_ERR_ARG = 1,        /* invalid argument or size                         */
  WC4D_ERR_NOT_SPD = 2,    /* Cholesky met a non-positive pivot                */
  WC4D_ERR_NONFINITE = 3,  /* NaN/Inf in inputs or Krylov scalars              */
  WC4D_ERR_BREAKDOWN = 4,  /* Lanczos/Arnoldi breakdown before convergence     */
  WC4D_ERR_MAXIT = 5,      /* tolerance not reached within maxit iterations    */
  WC4D_ERR_TIMEOUT = 6,    /* a bounded device wait gave up (wc4d_status)      */
  WC4D_ERR_CUDA = 7,       /* CUDA runtime error                               */
  WC4D_ERR_NOMEM = 8,      /* device allocation failed                         */
  WC4D_ERR_IO = 9          /* checkpoint file could not be read or written     */
};

/* model operator M_i (Eq. def:L) */
enum {
  WC4D_MODEL_STENCIL3 = 0, /* (M x)_j = c0 x_{j-1} + c1 x_j + c2 x_{j+1}, periodic, same for all i */
  WC4D_MODEL_BANDED = 1    /* per-time banded M_i, offsets -band_lo..band_hi, periodic wrap        */
};
/* covariance source */
enum {
  WC4D_COV_DENSE = 0,      /* caller passes dense B (s x s), Q (s x s), R (p x p)                   */
  WC4D_COV_SOAR = 1,       /* library builds SOAR matrices on the device (Sec. 6.1, Eq. SOAR):
                              c(r) = sigma2 (1 + r/ell) exp(-r/ell), r = chordal distance between
                              points x_j = j/s of the periodic unit domain, r = sin(pi |dx|)/pi;
                              R uses the observed points x = obs_idx/s                              */
  WC4D_COV_MSOAR = 2       /* B and Q are the banded circulant "modified SOAR" of the heat-equation
                              experiments (Sec. 6.1): first row c_i = amp (1 + d_i/L) exp(-d_i/L),
                              d_i = 2 |sin(i theta / 2)|, theta = pi / maxval, for |i| <= maxval and
                              zero beyond, plus delta I with delta = |lambda_min| + psi when the
                              circulant has a negative eigenvalue (lambda from the DFT of the row);
                              (amp, L, maxval) in msoar_b / msoar_q, psi in msoar_psi.  B and Q are
                              never formed: their products run through the band (2 maxval + 1 taps
                              per output).  R is the caller's dense R when R != NULL, else the SOAR
                              over the observed points (soar_r).  Needs precond PI (no Dhat^-1 of
                              a band), shat PAPER, covprod DENSE, one observation set             */
};
enum { WC4D_MEM_HOST = 0, WC4D_MEM_DEVICE = 1 };

enum { WC4D_PRECOND_PD = 0, WC4D_PRECOND_PI = 1 };          /* Eq. prec                     */
enum { WC4D_RHAT_EXACT = 0, WC4D_RHAT_RR = 1,               /* Rhat = R; Alg. 1 ridge       */
       WC4D_RHAT_ME = 2, WC4D_RHAT_DIAG = 3,                /* Alg. 2 min-eig; Sec. 5.1     */
       WC4D_RHAT_BLOCK = 4 };     /* Alg. 3 (Sec. 5.1): R's channel blocks (rblock_sizes) are
                                     decoupled where the first super-diagonal block's Frobenius
                                     norm over sqrt(size_j size_j+1) is below rblock_tol; Rhat
                                     keeps R inside each run of coupled blocks (every level) and
                                     is zero between runs.  Optional size / count rules: a run
                                     above rblock_maxsize rows is cut at its row midpoint; more
                                     runs than rblock_numproc joins the adjacent pair with the
                                     smallest total size, fewer than rblock_numproc - 2 cuts the
                                     largest run at its midpoint (ties: the first); each rule
                                     applies once, in this order                                */
enum { WC4D_LHAT_LM = 0,          /* Lhat = L_M(k) with the model's M_i (Definition 1)          */
       WC4D_LHAT_I = 1 };         /* Lhat = L_I (Sec. 2.2): every M_i inside Lhat replaced by the
                                     identity, chunked by k like L_M(k) (k = N+1: the printed
                                     L_I); the saddle matrix keeps M                            */
enum { WC4D_SHAT_PAPER = 0, WC4D_SHAT_EXACT = 1,           /* Lhat^T D^-1 Lhat ; S (Sec 2.2) */
       WC4D_SHAT_LEARNED = 2 };   /* PAPER plus a learned correction of its inverse (not in the
                                     paper; wc4d_precond_train / _load), GMRES only          */
enum { WC4D_DHAT_EXACT = 0, WC4D_DHAT_SHIFT = 1 };          /* D ; D + delta I (Sec. 6.1)   */
enum { WC4D_KRYLOV_MINRES = 0, WC4D_KRYLOV_GMRES = 1, WC4D_KRYLOV_FGMRES = 2 };
enum { WC4D_COVPROD_DENSE = 0,    /* B, Q as dense s x s products; Dhat^-1 through inverse Cholesky
                                     factors                                                    */
       WC4D_COVPROD_FFT = 1 };    /* B and Q are circulant (Sec. 6.1: SOAR on the periodic uniform
                                     grid depends on (i - j) mod s only): B v, Q v, Bhat^-1 v and
                                     Qhat^-1 v as FP64 FFT, scaling by the real spectrum (or its
                                     inverse, with the Dhat shift) and inverse FFT; no s x s
                                     factorisation.  Needs s a power of two in [64, 8192],
                                     precision FP64, DF32 or OZAKI, shat PAPER or LEARNED; with
                                     cov_kind DENSE the caller's B and Q must be circulant
                                     (checked at setup: ARG otherwise), the spectrum being taken
                                     from their first columns.  A spectrum value <= 0 gives
                                     NOT_SPD.  R stays a dense product (the observed points are
                                     not a uniform grid).                                       */
enum { WC4D_TOEPLITZ_AUTO = 0, WC4D_TOEPLITZ_OFF = 1 };  /* wc4d_solve_opts.toeplitz_gemv */
enum { WC4D_PREC_FP64 = 0,        /* every product in native FP64 (DFMA)                       */
       WC4D_PREC_MIXED = 1,       /* FGMRES outer (FP64-accurate A) around an FP32 inner GMRES
                                     preconditioned by an FP32 copy of the chosen preconditioner
                                     (not in the paper)                                         */
       WC4D_PREC_DF32 = 2,        /* every covariance / factor product in double-float on the
                                     FP32 pipe (operands split into two FP32 parts, exact
                                     product errors, TwoSum accumulation: ~48-bit products);
                                     recurrences, dots, factorisations and the true residual
                                     stay FP64 (not in the paper)                               */
       WC4D_PREC_DF32_P32 = 3,    /* GMRES only: A and the Arnoldi process as in DF32, the
                                     preconditioner applied in FP32 (FP32 copies of the
                                     operators and factors).  The DF32 Arnoldi keeps the
                                     computed preconditioned vectors, so GMRES is flexible and
                                     the FP32 rounding of P^-1 costs iterations, not accuracy
                                     (not in the paper)                                         */
       WC4D_PREC_OZAKI = 4 };     /* as DF32, but every covariance / factor product with two or
                                     more right-hand sides runs on the tensor cores: operator
                                     rows and vector columns are cut into 7 balanced base-128
                                     digits (47 bits below a power-of-two scale per row /
                                     column), the 28 digit products of significance levels
                                     0..6 accumulate exactly in FP32 (K-ranges of at most 512)
                                     and are combined in double-float; one-column products run
                                     in double-float (Ozaki, Ogita, Oishi and Rump 2012; not in
                                     the paper)                                                 */

typedef struct {
  int32_t s;                 /* state size per time level, >= 2                         */
  int32_t N;                 /* number of subwindows; N+1 time levels, >= 0             */
  int32_t p;                 /* observations per time level, 1 <= p <= s                */
  int32_t model_kind;        /* WC4D_MODEL_*                                            */
  double stencil[3];         /* STENCIL3 coefficients (c0, c1, c2)                      */
  int32_t band_lo, band_hi;  /* BANDED: offsets; band_lo + band_hi + 1 <= s             */
  const double* bands;       /* BANDED: [N][s][band_lo+band_hi+1],
                                bands[i-1][j][o+band_lo] = (M_i)[j][(j+o) mod s];
                                may be NULL (all zero) when wc4d_l96_gauss_newton fills it */
  const int32_t* obs_idx;    /* [p] strictly increasing indices in [0, s)               */
  int32_t cov_kind;          /* WC4D_COV_*                                              */
  const double* B;           /* DENSE: s x s                                            */
  const double* Q;           /* DENSE: s x s                                            */
  const double* R;           /* DENSE: p x p                                            */
  double soar_b[2];          /* SOAR: (sigma2, ell) of B, ell as a fraction of the domain */
  double soar_q[2];          /* SOAR: (sigma2, ell) of Q                                */
  double soar_r[2];          /* SOAR: (sigma2, ell) of R                                */
  int32_t mem_kind;          /* where bands/obs_idx/B/Q/R live: WC4D_MEM_HOST|DEVICE    */
  double msoar_b[3];         /* MSOAR: (amp, L, maxval) of B, maxval integral, 2 maxval + 1 <= s */
  double msoar_q[3];         /* MSOAR: (amp, L, maxval) of Q                                */
  double msoar_psi[2];       /* MSOAR: the shifts' draws psi of B and Q (>= 0)              */
  const int32_t* p_t;        /* NULL: one set obs_idx[p] and one R (p x p) for every time
                                level (Sec. 6.1).  Else per-time observation sets (Sec. 2.1:
                                H = blkdiag(H_i), R = blkdiag(R_i)): host array of the N+1
                                counts p_0..p_N, each in [1, s], summing to p; obs_idx then
                                holds the N+1 strictly increasing sets one after another, a
                                DENSE R the N+1 blocks R_0..R_N (p_i x p_i each) one after
                                another, and SOAR builds each R_i over its own set.  In a
                                vector nu_i is p_i long and starts at p_0 + .. + p_{i-1}.
                                Each Rhat_i is built from R_i alone (rhat EXACT, DIAG, RR or
                                ME); needs shat PAPER and precision FP64, DF32 or OZAKI, and
                                is not available to wc4d_synthesize_rhs or the Lorenz-96
                                calls.  Read during setup only.                           */
} wc4d_problem_desc;

typedef struct {
  int32_t precond;           /* WC4D_PRECOND_PD (MINRES) or WC4D_PRECOND_PI (GMRES)        */
  int32_t k;                 /* Lhat = L_M(k), 1 <= k <= N+1; 1 gives L_0 = I, N+1 gives L */
  int32_t rhat;              /* WC4D_RHAT_*                                                 */
  double kappa_max;          /* Alg. 1 / Alg. 2 target condition number (> 1)               */
  int32_t shat;              /* WC4D_SHAT_*; EXACT needs s(N+1) <= 8192                     */
  int32_t dhat;              /* WC4D_DHAT_*                                                 */
  double dhat_delta;         /* SHIFT: Dhat = D + delta I                                   */
  int32_t krylov;            /* WC4D_KRYLOV_*                                               */
  double tol;                /* relative residual in the 2-norm (1e-6 in Sec. 7)            */
  int32_t maxit;             /* outer iteration cap (1000 in Sec. 7)                        */
  int32_t precision;         /* WC4D_PREC_*                                                 */
  int32_t inner_iters;       /* MIXED: inner GMRES steps per outer FGMRES step              */
  int32_t check_every;       /* host polls the device convergence flag every this many steps */
  int32_t lhat;              /* WC4D_LHAT_*                                                 */
  int32_t rblock_count;      /* RHAT_BLOCK: number of channel blocks (pvec of Alg. 3), >= 1 */
  const int32_t* rblock_sizes; /* RHAT_BLOCK: host array [rblock_count] of block sizes, each
                                  >= 1, summing to p; read during setup only (caller-owned)  */
  double rblock_tol;         /* RHAT_BLOCK: Alg. 3 tol (>= 0; infinity cuts every coupling)  */
  int32_t rblock_maxsize;    /* RHAT_BLOCK: Alg. 3 maxsize in rows; 0 = no size rule        */
  int32_t rblock_numproc;    /* RHAT_BLOCK: Alg. 3 numproc; 0 = no count rule              */
  int32_t covprod;           /* WC4D_COVPROD_*: how B, Q (and Bhat^-1, Qhat^-1) are applied */
  int32_t prec_digits;       /* OZAKI + GMRES: leading BF16 digits (1..7; 0 = 7) of each operand
                                in the preconditioner's tensor-core products.  7 digits keep the
                                47-bit operands (FP64-class); d < 7 digits is a reduced-precision
                                product of about 7d - 1 bits (d = 1: BF16 inputs, d = 3: about
                                FP32) that reads d/7 of the digit bytes and issues d(d+1)/2 of
                                the 28 digit products, with exact FP32 accumulation.  The GMRES
                                keeps the computed preconditioned vectors (flexible), so the
                                rounding costs iterations, not accuracy; A v, the Arnoldi process
                                and the true residual stay FP64-class (not in the paper).       */
  int32_t rinv_explicit;     /* 0: Rhat^-1 v = W^T (W v) with W = chol(Rhat)^-1, two dependent
                                products (Sec. 6.2's triangular solves as products); 1: the
                                symmetric inverse W^T W is formed once at setup and Rhat^-1 v is
                                one product, in the same launch as P_I's D c1 (the same bytes,
                                one dependency level less per preconditioner apply).  Needs one
                                observation set, precision FP64, DF32 or OZAKI, shat PAPER or
                                LEARNED (not in the paper)                                      */
  int32_t basis_bytes;       /* DF32 / OZAKI GMRES: bytes per entry of the stored Arnoldi basis.
                                0 or 8: double-float (FP32 high + FP32 low part, about 48
                                significant bits); 6: FP32 high + BF16 low part (about 32 bits),
                                a quarter fewer bytes in the two basis passes of every step.  The
                                stored basis rounding bounds the attainable true residual near
                                1e-9 relative: use 6 with tol >= 1e-7 (checked: WC4D_ERR_ARG
                                otherwise).  Any other value is WC4D_ERR_ARG (not in the paper) */
  int32_t toeplitz_gemv;     /* OZAKI: WC4D_TOEPLITZ_AUTO (0, the default) or WC4D_TOEPLITZ_OFF.
                                AUTO: when B (Q) is symmetric Toeplitz -- every entry bitwise equal
                                to its first row's entry at |i - j|, as the SOAR covariances of the
                                periodic uniform grid (Sec. 6.1) that WC4D_COV_SOAR builds -- its
                                one-column products (B on time level 0; Q on a single or a 65th
                                column) read the split first row instead of the s x s entries: the
                                same operand values in the same order, so bitwise the same result,
                                from 8 s instead of 8 s^2 bytes.  Checked once at setup; any other
                                operator, or OFF, reads the dense rows.  Other values: ARG       */
} wc4d_solve_opts;

typedef struct {
  int32_t status;            /* WC4D_OK or the failure code                              */
  int32_t iters;             /* outer Krylov iterations                                  */
  int32_t inner_iters;       /* MIXED: total inner iterations                            */
  int32_t precond_fallback;  /* SHAT_LEARNED: 1 if the solve with the learned Schur block
                                failed and was repeated with the plain one (the reported
                                fields are the repeated solve's)                         */
  double relres_true;        /* ||rhs - A x||_2 / ||rhs||_2 recomputed in FP64 at exit   */
  double relres_est;         /* recurrence estimate at exit                              */
  double ms;                 /* wall time of the solve call                              */
  int64_t n_apply_A;         /* FP64 applications of A                                   */
  int64_t n_apply_P;         /* applications of the preconditioner (any precision)      */
  /* Per-component product counts in the convention of Tables 4 and 5 (Sec. 7):
   * one count per time block a product touches, so a full pass over the
   * window counts N+1.  Per A v: N+1 R_i, N+1 D_i and 2N model products
   * (L v3, L^T v1).  Per P_D^{-1} v: N+1 Dhat_i^{-1}, N+1 Rhat_i^{-1}, N+1 D_i
   * (Shat^{-1} = Lhat^{-1} D Lhat^{-T}) and 2 (N - floor(N/k)) model products
   * in the two Lhat sweeps (none with the exact S or with Lhat = L_I).  Per
   * P_I^{-1} v: N+1 Rhat_i^{-1}, N+1 D_i (D c1) and the same sweep products.
   * The mixed mode counts its inner FP32 A and P applies.                      */
  int64_t n_cov;             /* covariance products: n_R + n_D                          */
  int64_t n_M;               /* model products M_i v and M_i^T v                        */
  int64_t n_trsm;            /* inverse-covariance applies: n_Dhat_inv + n_Rhat_inv    */
  int64_t n_R, n_D, n_Dhat_inv, n_Rhat_inv;  /* n_cov and n_trsm by operator          */
} wc4d_info;

typedef struct wc4d_problem wc4d_problem;   /* opaque, library-owned */

/* Fill opts with the defaults of Sec. 7: P_I + GMRES, k = 1, Lhat = L_M(k),
 * Rhat = R, kappa_max = 100, paper Shat, exact Dhat, tol 1e-6, maxit 1000,
 * FP64; the Alg. 3 fields zero (no channel blocks). */
void wc4d_default_opts(wc4d_solve_opts* opts);

/* Build a problem: copy/generate B, Q, R, M_i and H on the device, build
 * Rhat (Alg. 1/2/3 or Sec. 5.1), factor Dhat, Rhat (and S when requested) with
 * FP64 Cholesky, invert the triangular factors, and allocate the Krylov
 * workspace for opts->maxit iterations.  cuda_stream is a cudaStream_t (NULL =
 * legacy default stream).  On success *out owns all device memory it uses;
 * release it with wc4d_destroy.  Errors: ARG (sizes, indices, options),
 * NOT_SPD (Cholesky of Dhat/Rhat/S failed), NONFINITE, NOMEM, CUDA.
 * Synchronises the stream before returning. */
int wc4d_setup_problem(const wc4d_problem_desc* desc, const wc4d_solve_opts* opts,
                       void* cuda_stream, wc4d_problem** out);

/* out = A v (Sec. 6.2: c1 = D v1 + L v3, c2 = R v2 + H v3, c3 = L^T v1 + H^T v2).
 * v, out: device, n doubles each, must not overlap.  Stream-ordered, async. */
int wc4d_apply_saddle(wc4d_problem* prob, const double* v, double* out);

/* Failure detection of the asynchronous calls.  In WC4D_PREC_OZAKI mode the
 * tensor-core product kernel runs a copy / MMA / epilogue pipeline whose
 * mbarrier waits are bounded (1 s by default); if one gives up, the kernel
 * stops writing, waits (again bounded) for its own copies and products, frees
 * its tensor memory and sets the problem's error word.  wc4d_solve reads and
 * clears that word after every solve and returns WC4D_ERR_TIMEOUT; after
 * wc4d_apply_saddle / wc4d_apply_precond (which only enqueue) call
 * wc4d_status: it synchronises the problem's stream, reads and clears the
 * word, and returns WC4D_ERR_TIMEOUT if a wait gave up (every output since
 * the previous check is then invalid), else WC4D_OK.  No counterpart in the
 * paper. */
int wc4d_status(wc4d_problem* prob);
/* Process-wide time limit of those pipeline waits in nanoseconds (0 restores
 * the default of 1 s), read at each launch.  The drain waits before a CTA
 * exits always keep the default.  For tests of the failure path: a limit of
 * a few ns makes a wait give up. */
void wc4d_set_wait_limit_ns(uint64_t ns);

/* out = P^{-1} v for which = WC4D_PRECOND_PD (Dhat^{-1} v1, Rhat^{-1} v2,
 * Lhat^{-1} D Lhat^{-T} v3, Sec. 6.2) or WC4D_PRECOND_PI (c1 = Lhat^{-T} v3,
 * c2 = Rhat^{-1} v2, c3 = Lhat^{-1}(v1 - D c1)).  P_D needs a problem set up
 * with opts->precond = PD (its Dhat factors); P_I is always available.
 * v, out: device, n doubles each, must not overlap.  Stream-ordered, async. */
int wc4d_apply_precond(wc4d_problem* prob, int32_t which, const double* v, double* out);

/* Solve A x = rhs with the Krylov method and preconditioner chosen at setup
 * (Sec. 6.2 / 7): MINRES for P_D, GMRES without restarts for P_I, FGMRES for
 * the mixed-precision mode.  rhs and x are FP64 vectors of length n, both on
 * the device (mem_kind = WC4D_MEM_DEVICE) or both on the host (HOST: copied
 * in and out through the problem's buffers).  x is the initial guess when
 * use_x0 != 0, otherwise it is ignored on input.  Blocks until the solution
 * is written.  info (may be NULL) receives iteration counts, residuals and
 * timings.  Returns MAXIT if the tolerance was not reached (x then holds the
 * last iterate), BREAKDOWN, NONFINITE or CUDA on failure. */
int wc4d_solve(wc4d_problem* prob, const double* rhs, double* x, int32_t use_x0,
               int32_t mem_kind, wc4d_info* info);

/* Batched solve of count independent problems (assimilation windows of any
 * s, N, p, model and precision, each set up by wc4d_setup_problem); not in the
 * paper, whose experiments solve one window at a time.  Equivalent to calling
 * wc4d_solve(probs[i], rhs[i], x[i], use_x0, mem_kind, &infos[i]) for every i,
 * but windows run concurrently: `workers` host threads (0 = min(count, 8),
 * at most 64) each own a non-blocking CUDA stream and take windows
 * largest-first by (s^2 + p^2)(N+1).  Each problem's own stream is
 * synchronised on entry (inputs produced on it are complete) and is restored
 * on return.  probs: distinct problems on the current device; rhs[i], x[i]:
 * n_i doubles each, all host or all device per mem_kind.  infos: NULL or
 * count entries.  Blocks until every window has finished.  Returns the status
 * of the lowest-indexed window that failed (its message names it), else OK.
 * Not for concurrent use with wc4d_set_profiling (single-stream profile). */
int wc4d_solve_batch(wc4d_problem* const* probs, int32_t count, const double* const* rhs, double* const* x,
                     int32_t use_x0, int32_t mem_kind, int32_t workers, wc4d_info* infos);

/* ---------------------------------------------------------------- learned
 * Learned Schur-block preconditioner (not in the paper).  P_D's third block
 * S_hat^{-1} = Lhat^{-1} D Lhat^{-T} (Sec. 2.2, Definition 1) gives y; the
 * learned block returns z = |y| (y/|y| + f(y/|y|)), f a 1D convolutional net
 * over the grid with the N+1 time levels as channels: conv(N+1 -> H) ReLU
 * conv(H -> H) ReLU conv(H -> H) ReLU conv(H -> N+1), kernel 5, periodic
 * 'same' padding, FP32.  It is trained to map y = S_hat^{-1} r to S^{-1} r,
 * S = L^T D^-1 L + H^T R^-1 H (the exact Schur complement): pairs are made
 * exactly by drawing v (white, or S_hat^{-1} of white noise, alternately),
 * forming r = S v with the problem's own operators, and t = v = S^{-1} r.
 * Needs a problem set up with precond = PD, shat = LEARNED, rhat = EXACT,
 * dhat = EXACT, krylov = GMRES (the net is nonlinear; the library's GMRES
 * keeps the preconditioned vectors and is therefore flexible), N + 1 <= 64.
 * The plain block (shat = PAPER) is the fallback and the yardstick: training
 * compares both on held-out pairs in the metric of the loss and activates the
 * net only if it is smaller; a solve that fails with the net is repeated
 * without it (wc4d_info.precond_fallback). */
typedef struct {
  int32_t pairs;             /* training + validation pairs generated (50000)       */
  int32_t hidden;            /* hidden channels H, <= 64 (32)                       */
  int32_t batch;             /* minibatch (64)                                      */
  int32_t epochs;            /* passes over the training pairs (4)                  */
  double lr;                 /* Adam step size (1e-3)                               */
  double val_frac;           /* held-out fraction (0.05)                            */
  uint64_t seed;             /* draws, initialisation and shuffling                 */
  int32_t loss;              /* WC4D_LOSS_*: what training minimises and the held-out
                                comparison uses (WC4D_LOSS_ERROR)                   */
} wc4d_train_opts;
enum { WC4D_LOSS_ERROR = 0,     /* |z - S^-1 r|^2 / |S^-1 r|^2: the error of the Schur solve */
       WC4D_LOSS_RESIDUAL = 1   /* |S z - r|^2 / |r|^2: the preconditioned residual, the
                                   quantity GMRES sees (two S applies per pair and step) */
};
typedef struct {
  double loss_first;         /* mean training loss |z - t|^2/|t|^2, first epoch     */
  double loss_last;          /* ... last epoch                                      */
  double val_err_learned;    /* held-out RMS of the loss's relative error, with the net */
  double val_err_plain;      /* ... with the plain S_hat^{-1} (z = y)               */
  int32_t kept;              /* 1 if the net is active (learned error < plain)      */
  int32_t pairs_train;       /* pairs used for training                             */
  double gen_ms, train_ms;   /* pair generation / training wall time                */
} wc4d_train_report;
void wc4d_default_train_opts(wc4d_train_opts* opts);
/* Generate pairs, train on the device, validate, and (ckpt_path != NULL) save
 * the weights.  report may be NULL.  Device memory: 8 (N+1) s bytes per pair
 * plus the problem's own.  Synchronises the stream.  Errors: ARG (problem not
 * set up as above, bad options), NOMEM, CUDA, IO (checkpoint file). */
int wc4d_precond_train(wc4d_problem* prob, const wc4d_train_opts* opts, const char* ckpt_path,
                       wc4d_train_report* report);
/* Load weights saved by wc4d_precond_train (same N+1 and s); the net is
 * activated if its saved validation error beat the plain block's. */
int wc4d_precond_load(wc4d_problem* prob, const char* ckpt_path);
/* Set the net's weights directly (host array, layout: for each layer l,
 * W[co][ci][5] then b[co]) and whether it is active. */
int wc4d_precond_set_net(wc4d_problem* prob, int32_t hidden, const float* params, int32_t active);
/* Mean loss and parameter gradients of the net on B host samples yn, tn
 * ([B][C][s] each, tn2 = |tn|^2 per sample), computed by the library's device
 * kernels; for checking them against a reference.  params, grads: host,
 * nparams floats. */
int wc4d_net_grad(int32_t C, int32_t hidden, int32_t s, int32_t B, const float* params, const float* yn,
                  const float* tn, double* loss, float* grads);
int64_t wc4d_net_nparams(int32_t C, int32_t hidden);

/* FP32 operators of the mixed-precision mode (not in the paper): out = A v
 * (which = 0), P_D^{-1} v (which = WC4D_PRECOND_PD + 1) or P_I^{-1} v
 * (which = WC4D_PRECOND_PI + 1), computed from FP32 copies of the covariances
 * and inverse factors with FP32 arithmetic (dot products in FP64).  v, out:
 * device, n floats each, not overlapping.  Needs a problem set up with
 * precision = WC4D_PREC_MIXED or WC4D_PREC_DF32_P32 (ARG otherwise).
 * Stream-ordered, async. */
int wc4d_apply_fp32(wc4d_problem* prob, int32_t which, const float* v, float* out);

/* Synthetic right-hand side (b, d, 0) of the first outer loop for a
 * STENCIL3 (linear) model, built on the device from standard-normal draws.
 * Follows the data-assimilation setting of Sec. 1 / Sec. 2.1: background
 * x_b = x_0^t + chol(B) z_b, truth x_i^t = M x_{i-1}^t (perfect model),
 * observations y_i = H x_i^t + chol(R) z_i, and the first linearisation
 * trajectory is the background forecast x^(0)_i = M x^(0)_{i-1}, x^(0)_0 = x_b.
 * Then b = 0 and d_i = y_i - H x^(0)_i = -H M^i chol(B) z_b + chol(R) z_i
 * (the truth cancels for a linear model, so it is not an argument).
 * z_b: s doubles; z_r: (N+1) p doubles, time-major; rhs: n doubles out.  All
 * three on the host or all on the device per mem_kind.  Uses the problem's
 * B and R (not Rhat).  Synchronises the stream.  Errors: ARG (banded model),
 * NOT_SPD, NOMEM, CUDA. */
int wc4d_synthesize_rhs(wc4d_problem* prob, const double* z_b, const double* z_r, int32_t mem_kind, double* rhs);

/* Lorenz-96 incremental weak-constraint 4D-Var (Sec. 2.1, Sec. 7.1).
 * The problem must be set up with model_kind = WC4D_MODEL_BANDED,
 * band_lo = 8 * steps_per_obs and band_hi = 4 * steps_per_obs (the reach of
 * steps_per_obs RK4 steps of dx_j/dt = (x_{j+1} - x_{j-2}) x_{j-1} - x_j + F);
 * its bands may be NULL at setup (they are rebuilt here).  Each outer loop l:
 * M_t = exact Jacobian of the RK4 steps about x^(l)_{t-1} (banded),
 * b_0 = x_b - x^(l)_0, b_t = M_t(x^(l)_{t-1}) - x^(l)_t (nonlinear forecast),
 * d_t = y_t - H x^(l)_t, solve the saddle-point system with the set-up
 * Krylov method / preconditioner, x^(l+1) = x^(l) + dx.  B, Q, R and their
 * factors are reused across loops.
 *   xb: s doubles; y: (N+1) p doubles (time-major); traj: (N+1) s doubles,
 *   in: the initial trajectory when init_background = 0 (else ignored and
 *   replaced by the background forecast from xb), out: the final trajectory;
 *   all three host or all device per mem_kind.
 *   loop_info: NULL or outer_loops entries, one per inner solve.
 * Limits: s <= 4096 (the state and its tangent live in shared memory).
 * Returns the first failing inner solve's status (the loop stops there).
 * Synchronises the stream. */
typedef struct {
  double forcing;            /* F (8 in Sec. 7.1)                    */
  double dt;                 /* RK4 step                             */
  int32_t steps_per_obs;     /* RK4 steps between observation times  */
  int32_t outer_loops;       /* Gauss-Newton iterations              */
} wc4d_l96_params;
int wc4d_l96_gauss_newton(wc4d_problem* prob, const wc4d_l96_params* prm, const double* xb, const double* y,
                          double* traj, int32_t init_background, int32_t mem_kind, wc4d_info* loop_info);

/* The linearisation half of one Gauss-Newton outer loop: rebuild the
 * problem's banded M_t about traj (Jacobians of the RK4 steps) and write the
 * right-hand side (b, d, 0) about traj into rhs (n doubles).  Same
 * requirements and layouts as wc4d_l96_gauss_newton; xb, y, traj, rhs all host
 * or all device per mem_kind.  Synchronises the stream. */
int wc4d_l96_linearize(wc4d_problem* prob, const wc4d_l96_params* prm, const double* xb, const double* y,
                       const double* traj, int32_t mem_kind, double* rhs);

/* Problem sizes: n (vector length), s, N, p (with per-time sets: the sum of p_i). */
int wc4d_problem_dims(const wc4d_problem* prob, int64_t* n, int32_t* s, int32_t* N, int32_t* p);

/* Copy a library-built covariance (which = 0: B, 1: Q, 2: R, 3: Rhat) into
 * dst (device, col-major, s*s or p*p doubles; with per-time sets, R and Rhat
 * are the N+1 blocks one after another, sum of p_i^2 doubles).  For tests and
 * diagnostics. */
int wc4d_get_matrix(wc4d_problem* prob, int32_t which, double* dst);

/* Rhat parameter used at setup: gamma (Alg. 1), T (Alg. 2) or the number of
 * decoupled runs of channel blocks (Alg. 3); 0 otherwise. */
double wc4d_rhat_param(const wc4d_problem* prob);

/* Process-wide counters for measurement (no counterpart in the paper).
 * launches: kernels the library launched since the last reset.  With
 * profiling enabled the library also brackets every launch of its dominant
 * kernel classes with CUDA events on the launching stream: the covariance /
 * factor products (stream-K GEMM in FP64, FP32 and double-float, and the
 * tensor-core Ozaki products; work = algorithmic FLOPs: 2 x multiply-adds
 * over the non-zero triangle, plus bytes and BF16 MMA flops for the
 * tensor-core class) and the Arnoldi orthogonalisation passes (work = bytes
 * the pass must read and write); launches that exit early on a solve that has
 * already converged are not counted.  The events add stream operations
 * between launches (they also stop consecutive kernels from overlapping their
 * launch), so a timing of whole solves should be taken with profiling off.
 * wc4d_set_profiling(1) allocates and clears the flag buffer (synchronous);
 * wc4d_reset_stats and wc4d_get_stats synchronise the device.  Not
 * thread-safe across concurrent solves. */
typedef struct {
  int64_t launches;
  double gemm_ms, gemm_flops;
  int64_t gemm_launches;
  double orth_ms, orth_bytes;
  int64_t orth_launches;
  double gemm32_ms, gemm32_flops;
  int64_t gemm32_launches;
  double gemmdf_ms, gemmdf_flops;   /* double-float (WC4D_PREC_DF32) products */
  int64_t gemmdf_launches;
  double gemmtc_ms, gemmtc_flops;   /* Ozaki tensor-core (WC4D_PREC_OZAKI) products; flops as above */
  double gemmtc_bytes;              /* bytes those launches must move: operator digit tiles and GEMV
                                       operands read once, vector digit tiles once per product,
                                       partial tiles written                                       */
  double gemmtc_mma_flops;          /* BF16 tensor-core flops of the digit products issued         */
  int64_t gemmtc_launches;
  double gemmtc_alg_bytes;          /* the same launches' floor: each FP64 operator entry (its
                                       triangle for factors) read once, vectors read and written once */
  double circ_ms, circ_flops;       /* circulant FFT products (WC4D_COVPROD_FFT): FP64 flops counted
                                       as 5 s log2 s per complex transform (two per column pair) plus
                                       the spectrum scaling                                          */
  double circ_bytes;                /* input columns read and output columns written (+ epilogue
                                       operands)                                                    */
  int64_t circ_launches;
  double pt_ms, pt_bytes;           /* per-time R-family products: operator blocks (their triangle
                                       for factors) read once, vectors read and written             */
  int64_t pt_launches;
  double orth_moved_bytes;          /* bytes the Arnoldi passes counted in orth_bytes actually move:
                                       orth_bytes counts 8 B per basis entry (the FP64-equivalent
                                       floor); with basis_bytes = 6 the passes move 6 B per entry   */
} wc4d_stats;
void wc4d_set_profiling(int32_t enable);
void wc4d_reset_stats(void);
int wc4d_get_stats(wc4d_stats* out);

/* A v without any device allocation.  The paper has no counterpart: this is
 * for callers that cannot call cudaMalloc -- a thread sharing the GPU with a
 * framework whose caching allocator already holds nearly all device memory,
 * or a latency-critical loop that cannot pay for cudaMalloc/cudaFree, which may
 * synchronise the device.  It computes the same product as wc4d_apply_saddle
 * for a STENCIL3 model (c1 = D v1 + L v3, c2 = R v2 + H v3,
 * c3 = L^T v1 + H^T v2) from caller-owned device arrays and needs no problem
 * handle.
 *   stencil: host, 3 doubles (c0, c1, c2) of the periodic model step;
 *   obs_idx: device, p strictly increasing indices in [0, s);
 *   B, Q: device, s x s; R: device, p x p (symmetric, column-major);
 *   v, out: device, n = (2s+p)(N+1) doubles each, not overlapping;
 *   cuda_stream: cudaStream_t (NULL = legacy default stream); the call is
 *   stream-ordered and returns after enqueueing.
 * Scratch (split-K partial tiles and the inverse observation map) lives in
 * one 8 MiB file-scope device array that every GPU loading the library keeps
 * until the process exits.  Limits: s <= 131072 and at most 240 partial
 * 64x64 tiles, i.e. ceil(s/64)*(1 + ceil(N/64)) + ceil(p/64)*ceil((N+1)/64)
 * <= 240 (s = 2048, N = 64, p = 1024 needs 96); larger problems return
 * WC4D_ERR_ARG with a message and launch nothing.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  Every call reuses
 * the same array and overwrites it (nothing in it needs to start at zero), so
 * calls that overlap on the GPU -- on different streams, or from different
 * host threads -- race and must be serialised by the caller.  Observation
 * indices outside [0, s) are skipped (their c2 rows become NaN); other input
 * errors are not detected. */
int wc4d_apply_saddle_noalloc(int32_t s, int32_t N, int32_t p, const double* stencil, const int32_t* obs_idx,
                              const double* B, const double* Q, const double* R, const double* v, double* out,
                              void* cuda_stream);

void wc4d_destroy(wc4d_problem* prob);
const char* wc4d_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* WC4D_H */
