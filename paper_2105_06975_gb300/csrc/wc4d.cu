// wc4d C ABI: problem setup, the saddle-point operator A (Eq. saddlepointA),
// the preconditioners P_D and P_I (Eq. prec, applied as in Sec. 6.2) and the
// device-resident MINRES / GMRES / FGMRES drivers.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <string>
#include <fstream>
#include <random>
#include <thread>
#include <type_traits>
#include <vector>

#include "circulant.cuh"
#include "common.cuh"
#include "krylov.cuh"
#include "learned.cuh"
#include "ozaki.cuh"
#include "pertime.cuh"
#include "rblock.h"

namespace wc4d {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

template <typename T>
void lhat_sweep(const ModelDev& md, int k, const T* v, T* z, bool transpose, bool identity_model, const int* done,
                cudaStream_t st);
template <typename T>
void saddle_c3(const ModelDev& md, const T* v1, const T* v2, const int* inv, int p, T* c3, const int* done,
               cudaStream_t st);
void saddle_c3_split(const ModelDev& md, const double* v1, const double* v2, const int* inv, int p, double* c3,
                     float* c3h, float* c3l, const int* done, cudaStream_t st);
void saddle_c3_pertime(const ModelDev& md, const double* v1, const double* v2, const int* inv_all, const int* nuoff,
                       double* c3, float* c3h, float* c3l, const int* done, cudaStream_t st);

// Operator data in one precision: covariances, inverse Cholesky factors and
// the GEMM partial buffer.
struct Split {
  const float* h = nullptr;
  const float* l = nullptr;
};
struct Digits {  // Ozaki digit tiles and row scales of an operator
  const uint16_t* d = nullptr;
  const float* s = nullptr;
};
template <typename T>
struct OpSet {
  T *B = nullptr, *Q = nullptr, *R = nullptr;
  T *WB = nullptr, *WBt = nullptr, *WQ = nullptr, *WQt = nullptr, *WR = nullptr, *WRt = nullptr;
  T *WS = nullptr, *WSt = nullptr;
  T* Rinv = nullptr;  // explicit Rhat^-1 = W_R^T W_R (wc4d_solve_opts.rinv_explicit)
  T* partial = nullptr;
  T *t1 = nullptr, *t2 = nullptr, *t3 = nullptr;  // n-length scratch
  // double-float splits of the operators above (DF32 / MIXED outer products)
  int df32 = 0;
  std::vector<std::pair<const T*, Split>> splits;
  Split split_of(const T* m) const {
    for (auto& s : splits)
      if (s.first == m) return s.second;
    return Split{};
  }
  float *xh = nullptr, *xl = nullptr;  // split X operands of one launch (2 n floats each)
  int64_t xcap = 0;
  // OZAKI: wide products on the tensor cores from digit forms of the operators
  // and of each launch's X blocks; one-column products read the splits above
  int tc = 0;
  std::vector<std::pair<const T*, Digits>> digits;
  Digits digits_of(const T* m) const {
    for (auto& d : digits)
      if (d.first == m) return d.second;
    return Digits{};
  }
  // symmetric Toeplitz operators (B, Q): copies of the split first row that
  // their one-column products read instead of the s x s split
  std::vector<std::pair<const T*, Split>> toeps;
  Split toep_of(const T* m) const {
    for (auto& t : toeps)
      if (t.first == m) return t.second;
    return Split{};
  }
  std::vector<const T*> toep_tiled;  // operators whose digit tiles are shared by offset
  bool tiles_shared(const T* m) const { return std::find(toep_tiled.begin(), toep_tiled.end(), m) != toep_tiled.end(); }
  uint16_t* xd = nullptr;
  int64_t xdcap = 0;
  float* xs = nullptr;
  int64_t xscap = 0;
  float* xg = nullptr;  // double-float split of each op's GEMV column
  int64_t xgcap = 0;
  int* tc_err = nullptr;
  void attach_tc(GemmOpsT<T>& ops, cudaStream_t st) const {
    if constexpr (sizeof(T) == 8) {
      ops.tc = 1;
      ops.df32 = 1;
      ops.err = tc_err;
      ops.wait_ns = oz_wait_limit();
      OzColJobs jobs{};
      int64_t xoff = 0, soff = 0;
      int ctas = 0;
      int64_t goff = 0;
      for (int o = 0; o < ops.nops; ++o) {
        GemmOpT<T>& op = ops.op[o];
        const Split sp = split_of(op.At);
        op.Ah = sp.h;
        op.Al = sp.l;
        const int wide = oz_wide_tiles(op.ncols);
        const int gcol = oz_gemv_col(op.ncols);
        if ((wide == 0 && gcol < 0) || op.m <= 0 || op.kdim <= 0) continue;
        OzColJob& jb = jobs.j[jobs.n];
        jb = OzColJob{};
        jb.X = op.X;
        jb.ldx = op.ldx;
        jb.kdim = op.kdim;
        jb.ncols = op.ncols;
        jb.nkb = (op.kdim + OZ_BK - 1) / OZ_BK;
        jb.wide = wide;
        jb.gemv_col = gcol;
        if (wide > 0) {
          const Digits dg = digits_of(op.At);
          if (!dg.d) throw Error{WC4D_ERR_ARG, "internal: no digit form for a tensor-core operator"};
          op.Ad = dg.d;
          op.As = dg.s;
          op.toep_tiles = (tiles_shared(op.At) && op.lda == op.m && op.kdim == op.m && op.tri == TRI_FULL) ? 1 : 0;
          const int64_t xe = oz_x_elems(op.kdim, op.ncols);
          if (xoff + xe > xdcap || soff + (int64_t)wide * OZ_BN > xscap)
            throw Error{WC4D_ERR_ARG, "internal: digit operand buffer too small"};
          op.Xd = xd + xoff;
          op.Xs = xs + soff;
          jb.Xd = op.Xd;
          jb.Xs = op.Xs;
          xoff += xe;
          soff += (int64_t)wide * OZ_BN;
        }
        if (gcol >= 0) {
          if (!sp.h) throw Error{WC4D_ERR_ARG, "internal: no double-float split for a GEMV operator"};
          const int64_t ge = (op.kdim + 3) / 4 * 4;  // keep each part 16-byte aligned
          if (goff + 2 * ge > xgcap) throw Error{WC4D_ERR_ARG, "internal: GEMV operand buffer too small"};
          jb.Xgh = xg + goff;
          jb.Xgl = xg + goff + ge;
          op.Xh = jb.Xgh;
          op.Xl = jb.Xgl;
          goff += 2 * ge;
          const Split tp = toep_of(op.At);
          if (tp.h && op.lda == op.m && op.kdim == op.m && op.tri == TRI_FULL) {
            op.Th = tp.h;
            op.Tl = tp.l;
            op.toff = oz_toeplitz_off(op.m);
            op.tstride = oz_toeplitz_stride(op.m);
          }
        }
        jobs.cta_base[jobs.n] = ctas;
        ++jobs.n;
        ctas += wide * OZ_BN + (gcol >= 0 ? oz_gemv_ctas(op.kdim) : 0);
      }
      jobs.cta_base[jobs.n] = ctas;
      launch_oz_cols(jobs, st);
    }
  }
  // route every product of a launch through the double-float kernel: attach
  // the operator splits and split each op's X block once
  void attach(GemmOpsT<T>& ops, cudaStream_t st) const {
    if (tc) {
      attach_tc(ops, st);
      return;
    }
    if (!df32) return;
    ops.df32 = 1;
    int64_t off = 0;
    SplitBlocks sb{};
    for (int o = 0; o < ops.nops; ++o) {
      GemmOpT<T>& op = ops.op[o];
      const Split sp = split_of(op.At);
      op.Ah = sp.h;
      op.Al = sp.l;
      const int64_t cnt = (int64_t)op.m * op.ncols;
      if (cnt <= 0) continue;
      if (off + cnt > xcap) throw Error{WC4D_ERR_ARG, "internal: double-float operand buffer too small"};
      if constexpr (sizeof(T) == 8) {
        sb.a[sb.n] = op.X;
        sb.ld[sb.n] = op.ldx;
        sb.m[sb.n] = op.m;
        sb.off[sb.n] = (int)off;
        ++sb.n;
      }
      op.Xh = xh + off;
      op.Xl = xl + off;
      off += cnt;
    }
    if constexpr (sizeof(T) == 8) {  // one split launch for all operand blocks
      sb.off[sb.n] = (int)off;
      sb.total = (int)off;
      launch_split_df_multi(sb, xh, xl, st);
    }
  }
};

}  // namespace wc4d

using namespace wc4d;

namespace wc4d {
// Small pinned host blocks (status words, scalars) from a process-wide free
// list: cudaMallocHost / cudaFreeHost per problem cost more than a setup's
// kernels and cudaFreeHost synchronises the device.
constexpr size_t PINNED_BLOCK = 256;
constexpr int SETUP_FLAGS = 20;  // setup flag slots (device ints), read back through one pinned block
static_assert(sizeof(int) * SETUP_FLAGS <= PINNED_BLOCK, "setup flags exceed the pinned block");
inline std::mutex& pinned_mu() {
  static std::mutex m;
  return m;
}
inline std::vector<void*>& pinned_free_list() {
  static std::vector<void*> v;
  return v;
}
inline void* pinned_get() {
  {
    std::lock_guard<std::mutex> lk(pinned_mu());
    auto& v = pinned_free_list();
    if (!v.empty()) {
      void* p = v.back();
      v.pop_back();
      return p;
    }
  }
  void* p = nullptr;
  WC4D_CUDA(cudaMallocHost(&p, PINNED_BLOCK));
  return p;
}
inline void pinned_put(void* p) {
  std::lock_guard<std::mutex> lk(pinned_mu());
  pinned_free_list().push_back(p);
}

// The default memory pool of the current device retains freed blocks up to
// this many bytes (set once per device; process-local, not a GPU setting).
inline void retain_default_pool() {
  static std::mutex mu;
  static bool set[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lk(mu);
  if (set[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = 32ull << 30;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  set[dev] = true;
}
}  // namespace wc4d

struct wc4d_problem {
  int s = 0, N = 0, p = 0;
  int64_t n = 0, ns = 0, np = 0;
  cudaStream_t st = nullptr;
  wc4d_solve_opts o{};
  ModelDev md{};
  int *d_obs = nullptr, *d_inv = nullptr;
  double* d_bands = nullptr;
  double* d_Rhat = nullptr;
  double rhat_param = 0.0;
  std::vector<int> rblock_sizes;  // RHAT_BLOCK: channel block sizes (Alg. 3 pvec)
  int nS = 0;
  bool have_pd = false;
  OpSet<double> f64;
  OpSet<float> f32;  // MIXED: FP32 copies for the inner solve
  // WC4D_COVPROD_FFT: B and Q are circulant and applied by FFT (twiddle table,
  // spectra of B, Q and of Bhat^-1, Qhat^-1 in the FFT kernel's cluster layout)
  int pdig = 7;  // OZAKI: digits of the preconditioner's tensor-core products
  bool rinv = false;  // Rhat^-1 applied as one product with the explicit inverse
  // WC4D_COV_MSOAR: banded circulant B and Q, applied through their taps
  bool band = false;
  double *bandB = nullptr, *bandQ = nullptr;  // device, 2 mv + 1 taps each
  int mvB = 0, mvQ = 0;
  double deltaB = 0.0, deltaQ = 0.0;
  bool circ = false;
  double2* tw = nullptr;
  double *lamB = nullptr, *lamQ = nullptr, *lamBi = nullptr, *lamQi = nullptr;
  // DF32 / OZAKI: the transforms run in double-float (tables as (hi, lo) pairs)
  bool circ_df = false;
  float4* twdf = nullptr;
  float2 *lamBdf = nullptr, *lamQdf = nullptr, *lamBidf = nullptr, *lamQidf = nullptr;
  // per-time observation sets (desc.p_t): counts, device layout of the nu
  // blocks and of the R_i, Rhat_i, W_i = chol(Rhat_i)^-1 and W_i^T blocks
  // (one after another); the inverse maps are (N+1) x s
  bool pertime = false;
  std::vector<int> pt;
  PtLayout ptl{};
  int64_t pt_elems = 0;  // sum of p_i^2
  double *ptR = nullptr, *ptRh = nullptr, *ptW = nullptr, *ptWt = nullptr;
  GemmPlan plan_A, plan_pd1, plan_pd2, plan_pi1, plan_pi2;
  // MIXED inner GMRES(m) workspace (FP32 basis, FP64 Hessenberg/rotations)
  int mi = 0;
  float *Vi = nullptr, *Zi = nullptr, *stage = nullptr, *zf = nullptr;
  double *Hi = nullptr, *csi = nullptr, *sni = nullptr, *gi = nullptr, *yi = nullptr;
  double *h1i = nullptr, *h2i = nullptr, *hnexti = nullptr, *bnormi = nullptr, *parti = nullptr, *part2i = nullptr;
  DevStatus* stat_in = nullptr;
  int64_t inner_total = 0;
  // Krylov workspace
  int maxit = 0;
  double *V = nullptr, *Z = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr;
  double *h1 = nullptr, *h2 = nullptr, *hnext = nullptr, *bnorm = nullptr, *scal = nullptr;
  double *part = nullptr, *part2 = nullptr, *part3 = nullptr, *sc = nullptr;
  double *rhs = nullptr, *x = nullptr, *r = nullptr, *x0 = nullptr;
  // DF32 GMRES: Arnoldi basis stored split (hi/lo FP32), current vector and w in FP64
  bool split_basis = false;
  int64_t ldb = 0;  // leading dimension of the split basis
  float *Vh = nullptr, *Vl = nullptr, *wh = nullptr, *wl = nullptr;
  double *vcur = nullptr, *wbuf = nullptr;
  // DF32 GMRES with delayed reorthogonalisation: raw Hessenberg, scalar state,
  // previous b and c, update coefficients, reduced dot rows, operator scratch
  bool dcgs = false;
  bool b6 = false;  // delayed-CGS2 basis with BF16 low parts (6-byte entries)
  double *Hraw = nullptr, *Tm = nullptr, *dcst = nullptr, *bprev = nullptr, *cprev = nullptr, *ecoef = nullptr;
  double *red = nullptr, *yhat = nullptr, *hcbuf = nullptr;
  // learned Schur-block correction (shat = LEARNED): weights, inference scratch
  NetShape net_sh;
  float* net_params = nullptr;
  bool net_on = false;
  float *net_in = nullptr, *net_out = nullptr, *net_act[3] = {nullptr, nullptr, nullptr};
  double *net_nrm2 = nullptr, *net_part = nullptr;
  DevStatus* stat = nullptr;
  DevStatus* h_stat = nullptr;
  double* h_scal = nullptr;
  int* d_flags = nullptr;  // setup flag slots (see setup)
  int* d_kerr = nullptr;   // set by the tensor-core kernel if a bounded wait gave up (read after each solve)
  struct CholCheck {
    int64_t slot;
    const char* what;
    int m;
    bool spectrum = false;  // a circulant spectrum check instead of a Cholesky pivot
  };
  std::vector<CholCheck> chol_checks;
  struct ToepCheck {  // Toeplitz row copies of B or Q (or Q's shared digit tiles: rows.h == nullptr),
    const double* op;  // registered if the check's slot stays 0
    Split rows;
    int slot;
  };
  std::vector<ToepCheck> toep_checks;
  std::vector<void*> allocs;

  // Stream-ordered allocation from the device's default pool, which keeps up to
  // 32 GB of freed memory for reuse: building a problem again (a new window, or
  // a benchmark step) then costs no driver allocation of its workspace.
  template <typename T>
  T* alloc(int64_t count) {
    void* p = nullptr;
    if (count <= 0) count = 1;
    wc4d::retain_default_pool();
    cudaError_t e = cudaMallocAsync(&p, sizeof(T) * (size_t)count, st);
    if (e != cudaSuccess) throw Error{WC4D_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e)};
    allocs.push_back(p);
    return (T*)p;
  }
  ~wc4d_problem() {
    plan_free(plan_A);
    plan_free(plan_pd1);
    plan_free(plan_pd2);
    plan_free(plan_pi1);
    plan_free(plan_pi2);
    for (void* p : allocs) cudaFreeAsync(p, st);
    cudaStreamSynchronize(st);
    if (h_stat) pinned_put(h_stat);
    if (h_scal) pinned_put(h_scal);
  }
};

namespace wc4d {

static int max_gemm_ctas(bool df32 = false) { return gemm_resident_ctas(df32); }

// algorithmic bytes of one per-time product: each block (its triangle for the
// factors) read once, x read and the output written once (+ the gathered v3)
static double pt_bytes(const wc4d_problem* P, const PtProd& pr) {
  double a = 0.0;
  for (int pi : P->pt) a += (pr.tri == TRI_FULL) ? (double)pi * pi : 0.5 * (double)pi * (pi + 1);
  return 8.0 * (a + (double)P->np * (pr.mode == EPI_SADDLE_C2 ? 3 : 2));
}

// launch the circulant jobs in the problem's arithmetic: double-float
// transforms (and their spectrum tables) in the DF32 / OZAKI modes
static void run_circ(wc4d_problem* P, CircJobs& cj, const int* done) {
  cj.df = P->circ_df ? 1 : 0;
  if (cj.df) {
    for (int q = 0; q < cj.n; ++q) {
      const double* l = cj.j[q].lam;
      cj.j[q].lamdf = (l == P->lamB) ? P->lamBdf : (l == P->lamQ) ? P->lamQdf : (l == P->lamBi) ? P->lamBidf
                                                                                               : P->lamQidf;
    }
  }
  launch_circ(cj, P->s, P->tw, P->twdf, P->md, done, P->st);
}

// D x (B on column 0, Q on columns 1..N) off the product path, for circulant
// (FFT) or banded circulant (taps) B and Q, with the product epilogue: mode
// EPI_SADDLE_C1 (C_t = (D x)_t + (L v3)_t) or EPI_SUB_FROM (C = Y - D x)
static void d_offpath(wc4d_problem* P, const double* x, int mode, double* C, const double* v3, const double* Y,
                      float* Ch, float* Cl, const int* done) {
  const int s = P->s, N = P->N;
  const double* Y1 = Y ? Y + s : nullptr;
  if (P->circ) {
    CircJobs cj{};
    circ_add(cj, CircJob{x, s, 1, P->lamB, mode, C, s, 0, v3, Y, Ch, Cl});
    if (N > 0)
      circ_add(cj, CircJob{x + s, s, N, P->lamQ, mode, C + s, s, 1, v3, Y1, Ch ? Ch + s : nullptr,
                           Cl ? Cl + s : nullptr});
    run_circ(P, cj, done);
    return;
  }
  BandJobs bj{};
  bj.j[bj.n++] = BandJob{x, s, 1, P->bandB, P->mvB, P->deltaB, mode, C, s, 0, v3, Y, Ch, Cl};
  if (N > 0)
    bj.j[bj.n++] = BandJob{x + s, s, N, P->bandQ, P->mvQ, P->deltaQ, mode, C + s, s, 1, v3, Y1,
                           Ch ? Ch + s : nullptr, Cl ? Cl + s : nullptr};
  launch_band(bj, s, P->md, done, P->st);
}

// ------------------------------------------------------------ A v (Sec. 6.2)
// wh / wl (T = double, optional): also write the double-float split of out
template <typename T>
static void apply_A(wc4d_problem* P, OpSet<T>& os, const GemmPlan& plan, const T* v, T* out, const int* done,
                    float* wh = nullptr, float* wl = nullptr) {
  const int s = P->s, N = P->N, p = P->p;
  const T* v1 = v;
  const T* v2 = v + P->ns;
  const T* v3 = v + P->ns + P->np;
  T* c1 = out;
  T* c2 = out + P->ns;
  T* c3 = out + P->ns + P->np;
  const bool split = (sizeof(T) == 8) && wh != nullptr;
  if constexpr (sizeof(T) == 8) {
    if (P->pertime) {
      // c3 with each time's own set; D v1 + L v3 as usual; c2_t = R_t v2_t + H_t v3_t
      saddle_c3_pertime(P->md, v1, v2, P->d_inv, P->ptl.nuoff, c3, split ? wh + P->ns + P->np : nullptr,
                        split ? wl + P->ns + P->np : nullptr, done, P->st);
      if (P->circ || P->band) {
        d_offpath(P, v1, EPI_SADDLE_C1, c1, v3, nullptr, split ? wh : nullptr, split ? wl : nullptr, done);
      } else {
        GemmOpsT<T> ops{};
        EpisT<T> ep{};
        ops.nops = 2;
        ops.op[0] = {os.B, s, v1, s, s, s, 1, TRI_FULL};
        ops.op[1] = {os.Q, s, v1 + s, s, s, s, N, TRI_FULL};
        ep.e[0] = {EPI_SADDLE_C1, c1, s, 0, v3, nullptr};
        ep.e[1] = {EPI_SADDLE_C1, c1 + s, s, 1, v3, nullptr};
        if (split) {
          ep.e[0].Ch = wh;
          ep.e[0].Cl = wl;
          ep.e[1].Ch = wh + s;
          ep.e[1].Cl = wl + s;
        }
        os.attach(ops, P->st);
        gemm_run<T>(plan, ops, ep, os.partial, P->md, P->d_obs, done, P->st);
      }
      PtProd pr{};
      pr.A = P->ptR;
      pr.tri = TRI_FULL;
      pr.X = v2;
      pr.mode = EPI_SADDLE_C2;
      pr.C = c2;
      pr.v3 = v3;
      pr.Ch = split ? wh + P->ns : nullptr;
      pr.Cl = split ? wl + P->ns : nullptr;
      launch_pertime(P->ptl, pr, pt_bytes(P, pr), done, P->st);
      return;
    }
    if (split)
      saddle_c3_split(P->md, v1, v2, P->d_inv, p, c3, wh + P->ns + P->np, wl + P->ns + P->np, done, P->st);
    else
      saddle_c3<T>(P->md, v1, v2, P->d_inv, p, c3, done, P->st);
  } else {
    saddle_c3<T>(P->md, v1, v2, P->d_inv, p, c3, done, P->st);
  }
  if constexpr (sizeof(T) == 8) {
    if (P->circ || P->band) {
      // D v1 + L v3 by FFT or through the band, R v2 + H v3 on the product path
      d_offpath(P, v1, EPI_SADDLE_C1, c1, v3, nullptr, split ? wh : nullptr, split ? wl : nullptr, done);
      GemmOpsT<T> ops{};
      EpisT<T> ep{};
      ops.nops = 1;
      ops.op[0] = {os.R, p, v2, p, p, p, N + 1, TRI_FULL};
      ep.e[0] = {EPI_SADDLE_C2, c2, p, 0, v3, nullptr};
      if (split) {
        ep.e[0].Ch = wh + P->ns;
        ep.e[0].Cl = wl + P->ns;
      }
      os.attach(ops, P->st);
      gemm_run<T>(plan, ops, ep, os.partial, P->md, P->d_obs, done, P->st);
      return;
    }
  }
  GemmOpsT<T> ops{};
  EpisT<T> ep{};
  ops.nops = 3;
  ops.op[0] = {os.B, s, v1, s, s, s, 1, TRI_FULL};
  ops.op[1] = {os.Q, s, v1 + s, s, s, s, N, TRI_FULL};
  ops.op[2] = {os.R, p, v2, p, p, p, N + 1, TRI_FULL};
  ep.e[0] = {EPI_SADDLE_C1, c1, s, 0, v3, nullptr};
  ep.e[1] = {EPI_SADDLE_C1, c1 + s, s, 1, v3, nullptr};
  ep.e[2] = {EPI_SADDLE_C2, c2, p, 0, v3, nullptr};
  if (split) {
    ep.e[0].Ch = wh;
    ep.e[0].Cl = wl;
    ep.e[1].Ch = wh + s;
    ep.e[1].Cl = wl + s;
    ep.e[2].Ch = wh + P->ns;
    ep.e[2].Cl = wl + P->ns;
  }
  os.attach(ops, P->st);
  gemm_run<T>(plan, ops, ep, os.partial, P->md, P->d_obs, done, P->st);
}

// Learned correction of the third block, in place: y <- |y| (y/|y| + f(y/|y|)).
static void learned_block(wc4d_problem* P, double* y) {
  const int64_t len = (int64_t)(P->N + 1) * P->s;
  dot_partial<double>(y, y, len, P->net_part, nullptr, P->st);
  dot_finish(P->net_part, P->net_nrm2, 0, P->st);
  net_in_from(y, P->net_nrm2, P->net_in, len, P->st);
  float* acts[3] = {P->net_act[0], P->net_act[1], P->net_act[2]};
  net_forward(P->net_sh, P->net_params, 1, P->net_in, acts, P->net_out, P->st);
  net_out_to(P->net_in, P->net_out, P->net_nrm2, y, len, P->st);
}

// P_D^{-1} v = (Dhat^{-1} v1, Rhat^{-1} v2, Shat^{-1} v3); Dhat^{-1} = W^T W with
// W the inverse Cholesky factor, Shat^{-1} = Lhat^{-1} D Lhat^{-T} (paper) or
// W_S^T W_S (exact S).
template <typename T>
static void apply_PD(wc4d_problem* P, OpSet<T>& os, const GemmPlan& p1, const GemmPlan& p2, const T* v, T* out,
                     const int* done) {
  const int s = P->s, N = P->N, p = P->p, k = P->o.k;
  const bool ident = (P->o.lhat == WC4D_LHAT_I);
  const T* v1 = v;
  const T* v2 = v + P->ns;
  const T* v3 = v + P->ns + P->np;
  T* o1 = out;
  T* o2 = out + P->ns;
  T* o3 = out + P->ns + P->np;
  T* y1 = os.t1;             // W v1
  T* y2 = os.t1 + P->ns;     // W_R v2
  T* y3 = os.t2;             // Lhat^{-T} v3
  T* u3 = os.t3;             // D y3 (or W_S v3)
  const bool exactS = (P->o.shat == WC4D_SHAT_EXACT);
  if (!exactS) lhat_sweep<T>(P->md, k, v3, y3, true, ident, done, P->st);
  if constexpr (sizeof(T) == 8) {
    if (P->rinv && !exactS) {
      // Rhat^-1 v2 as one product with the explicit inverse
      GemmOpsT<T> ops{};
      EpisT<T> ep{};
      ops.ndig = P->pdig;
      ops.op[0] = {os.Rinv, p, v2, p, p, p, N + 1, TRI_FULL};
      ep.e[0] = {EPI_STORE, o2, p, 0, nullptr, nullptr};
      if (P->circ) {
        ops.nops = 1;
        os.attach(ops, P->st);
        gemm_run<T>(p1, ops, ep, os.partial, P->md, P->d_obs, done, P->st);
        CircJobs cj{};
        circ_add(cj, CircJob{v1, s, 1, P->lamBi, EPI_STORE, o1, s, 0, nullptr, nullptr});
        if (N > 0) circ_add(cj, CircJob{v1 + s, s, N, P->lamQi, EPI_STORE, o1 + s, s, 0, nullptr, nullptr});
        circ_add(cj, CircJob{y3, s, 1, P->lamB, EPI_STORE, u3, s, 0, nullptr, nullptr});
        if (N > 0) circ_add(cj, CircJob{y3 + s, s, N, P->lamQ, EPI_STORE, u3 + s, s, 0, nullptr, nullptr});
        run_circ(P, cj, done);
      } else {
        ops.nops = 4;
        ops.op[1] = {os.WBt, s, v1, s, s, s, 1, TRI_LOWER};
        ops.op[2] = {os.WQt, s, v1 + s, s, s, s, N, TRI_LOWER};
        ops.op[3] = {os.Q, s, y3 + s, s, s, s, N, TRI_FULL};
        ep.e[1] = {EPI_STORE, y1, s, 0, nullptr, nullptr};
        ep.e[2] = {EPI_STORE, y1 + s, s, 0, nullptr, nullptr};
        ep.e[3] = {EPI_STORE, u3 + s, s, 0, nullptr, nullptr};
        os.attach(ops, P->st);
        gemm_run<T>(p1, ops, ep, os.partial, P->md, P->d_obs, done, P->st);
        GemmOpsT<T> ops2{};
        EpisT<T> ep2{};
        ops2.nops = 3;
        ops2.ndig = P->pdig;
        ops2.op[0] = {os.WB, s, y1, s, s, s, 1, TRI_UPPER};
        ops2.op[1] = {os.WQ, s, y1 + s, s, s, s, N, TRI_UPPER};
        ops2.op[2] = {os.B, s, y3, s, s, s, 1, TRI_FULL};
        ep2.e[0] = {EPI_STORE, o1, s, 0, nullptr, nullptr};
        ep2.e[1] = {EPI_STORE, o1 + s, s, 0, nullptr, nullptr};
        ep2.e[2] = {EPI_STORE, u3, s, 0, nullptr, nullptr};
        os.attach(ops2, P->st);
        gemm_run<T>(p2, ops2, ep2, os.partial, P->md, P->d_obs, done, P->st);
      }
      lhat_sweep<T>(P->md, k, u3, o3, false, ident, done, P->st);
      if (P->net_on) learned_block(P, o3);
      return;
    }
    if (P->pertime) {
      // Rhat_t^{-1} v2_t = W_t^T (W_t v2_t) per time level; D parts as usual
      PtProd pr{};
      pr.A = P->ptWt;
      pr.tri = TRI_LOWER;
      pr.X = v2;
      pr.mode = EPI_STORE;
      pr.C = y2;
      launch_pertime(P->ptl, pr, pt_bytes(P, pr), done, P->st);
      if (P->circ) {
        CircJobs cj{};
        circ_add(cj, CircJob{v1, s, 1, P->lamBi, EPI_STORE, o1, s, 0, nullptr, nullptr});
        if (N > 0) circ_add(cj, CircJob{v1 + s, s, N, P->lamQi, EPI_STORE, o1 + s, s, 0, nullptr, nullptr});
        circ_add(cj, CircJob{y3, s, 1, P->lamB, EPI_STORE, u3, s, 0, nullptr, nullptr});
        if (N > 0) circ_add(cj, CircJob{y3 + s, s, N, P->lamQ, EPI_STORE, u3 + s, s, 0, nullptr, nullptr});
        run_circ(P, cj, done);
      } else {
        GemmOpsT<T> ops{};
        EpisT<T> ep{};
        ops.nops = 3;
        ops.ndig = P->pdig;
        ops.op[0] = {os.WBt, s, v1, s, s, s, 1, TRI_LOWER};
        ops.op[1] = {os.WQt, s, v1 + s, s, s, s, N, TRI_LOWER};
        ops.op[2] = {os.Q, s, y3 + s, s, s, s, N, TRI_FULL};
        ep.e[0] = {EPI_STORE, y1, s, 0, nullptr, nullptr};
        ep.e[1] = {EPI_STORE, y1 + s, s, 0, nullptr, nullptr};
        ep.e[2] = {EPI_STORE, u3 + s, s, 0, nullptr, nullptr};
        os.attach(ops, P->st);
        gemm_run<T>(p1, ops, ep, os.partial, P->md, P->d_obs, done, P->st);
        GemmOpsT<T> ops2{};
        EpisT<T> ep2{};
        ops2.nops = 3;
        ops2.ndig = P->pdig;
        ops2.op[0] = {os.WB, s, y1, s, s, s, 1, TRI_UPPER};
        ops2.op[1] = {os.WQ, s, y1 + s, s, s, s, N, TRI_UPPER};
        ops2.op[2] = {os.B, s, y3, s, s, s, 1, TRI_FULL};
        ep2.e[0] = {EPI_STORE, o1, s, 0, nullptr, nullptr};
        ep2.e[1] = {EPI_STORE, o1 + s, s, 0, nullptr, nullptr};
        ep2.e[2] = {EPI_STORE, u3, s, 0, nullptr, nullptr};
        os.attach(ops2, P->st);
        gemm_run<T>(p2, ops2, ep2, os.partial, P->md, P->d_obs, done, P->st);
      }
      PtProd pr2{};
      pr2.A = P->ptW;
      pr2.tri = TRI_UPPER;
      pr2.X = y2;
      pr2.mode = EPI_STORE;
      pr2.C = o2;
      launch_pertime(P->ptl, pr2, pt_bytes(P, pr2), done, P->st);
      lhat_sweep<T>(P->md, k, u3, o3, false, ident, done, P->st);
      return;
    }
    if (P->circ) {
      // Dhat^{-1} v1 and D y3 by FFT in one launch; Rhat^{-1} v2 = W^T (W v2)
      GemmOpsT<T> ops{};
      EpisT<T> ep{};
      ops.nops = 1;
      ops.ndig = P->pdig;
      ops.op[0] = {os.WRt, p, v2, p, p, p, N + 1, TRI_LOWER};
      ep.e[0] = {EPI_STORE, y2, p, 0, nullptr, nullptr};
      os.attach(ops, P->st);
      gemm_run<T>(p1, ops, ep, os.partial, P->md, P->d_obs, done, P->st);
      CircJobs cj{};
      circ_add(cj, CircJob{v1, s, 1, P->lamBi, EPI_STORE, o1, s, 0, nullptr, nullptr});
      if (N > 0) circ_add(cj, CircJob{v1 + s, s, N, P->lamQi, EPI_STORE, o1 + s, s, 0, nullptr, nullptr});
      circ_add(cj, CircJob{y3, s, 1, P->lamB, EPI_STORE, u3, s, 0, nullptr, nullptr});
      if (N > 0) circ_add(cj, CircJob{y3 + s, s, N, P->lamQ, EPI_STORE, u3 + s, s, 0, nullptr, nullptr});
      run_circ(P, cj, done);
      GemmOpsT<T> ops2{};
      EpisT<T> ep2{};
      ops2.nops = 1;
      ops2.ndig = P->pdig;
      ops2.op[0] = {os.WR, p, y2, p, p, p, N + 1, TRI_UPPER};
      ep2.e[0] = {EPI_STORE, o2, p, 0, nullptr, nullptr};
      os.attach(ops2, P->st);
      gemm_run<T>(p2, ops2, ep2, os.partial, P->md, P->d_obs, done, P->st);
      lhat_sweep<T>(P->md, k, u3, o3, false, ident, done, P->st);
      if (P->net_on) learned_block(P, o3);
      return;
    }
  }
  GemmOpsT<T> ops{};
  EpisT<T> ep{};
  ops.op[0] = {os.WBt, s, v1, s, s, s, 1, TRI_LOWER};
  ops.op[1] = {os.WQt, s, v1 + s, s, s, s, N, TRI_LOWER};
  ops.op[2] = {os.WRt, p, v2, p, p, p, N + 1, TRI_LOWER};
  ep.e[0] = {EPI_STORE, y1, s, 0, nullptr, nullptr};
  ep.e[1] = {EPI_STORE, y1 + s, s, 0, nullptr, nullptr};
  ep.e[2] = {EPI_STORE, y2, p, 0, nullptr, nullptr};
  if (exactS) {
    ops.nops = 4;
    ops.ndig = P->pdig;
    ops.op[3] = {os.WSt, P->nS, v3, P->nS, P->nS, P->nS, 1, TRI_LOWER};
    ep.e[3] = {EPI_STORE, u3, P->nS, 0, nullptr, nullptr};
  } else {
    ops.nops = 4;
    ops.ndig = P->pdig;
    // D y3 = [B y3_0 | Q y3_1..N]: two ops packed as one B-column op and one Q op
    // exceed GEMM_MAX_OPS together with the three factors, so B's column rides
    // in a second launch below.
    ops.op[3] = {os.Q, s, y3 + s, s, s, s, N, TRI_FULL};
    ep.e[3] = {EPI_STORE, u3 + s, s, 0, nullptr, nullptr};
  }
  os.attach(ops, P->st);
  gemm_run<T>(p1, ops, ep, os.partial, P->md, P->d_obs, done, P->st);
  GemmOpsT<T> ops2{};
  EpisT<T> ep2{};
  ops2.op[0] = {os.WB, s, y1, s, s, s, 1, TRI_UPPER};
  ops2.op[1] = {os.WQ, s, y1 + s, s, s, s, N, TRI_UPPER};
  ops2.op[2] = {os.WR, p, y2, p, p, p, N + 1, TRI_UPPER};
  ep2.e[0] = {EPI_STORE, o1, s, 0, nullptr, nullptr};
  ep2.e[1] = {EPI_STORE, o1 + s, s, 0, nullptr, nullptr};
  ep2.e[2] = {EPI_STORE, o2, p, 0, nullptr, nullptr};
  if (exactS) {
    ops2.nops = 4;
    ops2.ndig = P->pdig;
    ops2.op[3] = {os.WS, P->nS, u3, P->nS, P->nS, P->nS, 1, TRI_UPPER};
    ep2.e[3] = {EPI_STORE, o3, P->nS, 0, nullptr, nullptr};
    os.attach(ops2, P->st);
    gemm_run<T>(p2, ops2, ep2, os.partial, P->md, P->d_obs, done, P->st);
  } else {
    ops2.nops = 4;
    ops2.ndig = P->pdig;
    ops2.op[3] = {os.B, s, y3, s, s, s, 1, TRI_FULL};
    ep2.e[3] = {EPI_STORE, u3, s, 0, nullptr, nullptr};
    os.attach(ops2, P->st);
    gemm_run<T>(p2, ops2, ep2, os.partial, P->md, P->d_obs, done, P->st);
    lhat_sweep<T>(P->md, k, u3, o3, false, ident, done, P->st);
    if constexpr (std::is_same<T, double>::value) {
      if (P->net_on) learned_block(P, o3);
    }
  }
}

// P_I^{-1} v: c1 = Lhat^{-T} v3, c2 = Rhat^{-1} v2, c3 = Lhat^{-1}(v1 - D c1).
template <typename T>
static void apply_PI(wc4d_problem* P, OpSet<T>& os, const GemmPlan& p1, const GemmPlan& p2, const T* v, T* out,
                     const int* done) {
  const int s = P->s, N = P->N, p = P->p, k = P->o.k;
  const T* v1 = v;
  const T* v2 = v + P->ns;
  const T* v3 = v + P->ns + P->np;
  T* o1 = out;
  T* o2 = out + P->ns;
  T* o3 = out + P->ns + P->np;
  T* y2 = os.t1;  // W_R v2
  T* u = os.t2;   // v1 - D c1
  const bool ident = (P->o.lhat == WC4D_LHAT_I);
  lhat_sweep<T>(P->md, k, v3, o1, true, ident, done, P->st);
  if constexpr (sizeof(T) == 8) {
    if (P->rinv) {
      // Rhat^-1 v2 as one product with the explicit inverse, in the launch of D c1
      GemmOpsT<T> ops{};
      EpisT<T> ep{};
      ops.ndig = P->pdig;
      ops.op[0] = {os.Rinv, p, v2, p, p, p, N + 1, TRI_FULL};
      ep.e[0] = {EPI_STORE, o2, p, 0, nullptr, nullptr};
      if (P->circ || P->band) {
        ops.nops = 1;
      } else {
        ops.nops = 3;
        ops.op[1] = {os.B, s, o1, s, s, s, 1, TRI_FULL};
        ops.op[2] = {os.Q, s, o1 + s, s, s, s, N, TRI_FULL};
        ep.e[1] = {EPI_SUB_FROM, u, s, 0, nullptr, v1};
        ep.e[2] = {EPI_SUB_FROM, u + s, s, 0, nullptr, v1 + s};
      }
      os.attach(ops, P->st);
      gemm_run<T>(p1, ops, ep, os.partial, P->md, P->d_obs, done, P->st);
      if (P->circ || P->band) d_offpath(P, o1, EPI_SUB_FROM, u, nullptr, v1, nullptr, nullptr, done);
      lhat_sweep<T>(P->md, k, u, o3, false, ident, done, P->st);
      return;
    }
    if (P->pertime) {
      PtProd pr{};
      pr.A = P->ptWt;
      pr.tri = TRI_LOWER;
      pr.X = v2;
      pr.mode = EPI_STORE;
      pr.C = y2;
      launch_pertime(P->ptl, pr, pt_bytes(P, pr), done, P->st);
      if (P->circ || P->band) {
        d_offpath(P, o1, EPI_SUB_FROM, u, nullptr, v1, nullptr, nullptr, done);
      } else {
        GemmOpsT<T> ops{};
        EpisT<T> ep{};
        ops.nops = 2;
        ops.ndig = P->pdig;
        ops.op[0] = {os.B, s, o1, s, s, s, 1, TRI_FULL};
        ops.op[1] = {os.Q, s, o1 + s, s, s, s, N, TRI_FULL};
        ep.e[0] = {EPI_SUB_FROM, u, s, 0, nullptr, v1};
        ep.e[1] = {EPI_SUB_FROM, u + s, s, 0, nullptr, v1 + s};
        os.attach(ops, P->st);
        gemm_run<T>(p1, ops, ep, os.partial, P->md, P->d_obs, done, P->st);
      }
      PtProd pr2{};
      pr2.A = P->ptW;
      pr2.tri = TRI_UPPER;
      pr2.X = y2;
      pr2.mode = EPI_STORE;
      pr2.C = o2;
      launch_pertime(P->ptl, pr2, pt_bytes(P, pr2), done, P->st);
      lhat_sweep<T>(P->md, k, u, o3, false, ident, done, P->st);
      return;
    }
    if (P->circ || P->band) {
      GemmOpsT<T> ops{};
      EpisT<T> ep{};
      ops.nops = 1;
      ops.ndig = P->pdig;
      ops.op[0] = {os.WRt, p, v2, p, p, p, N + 1, TRI_LOWER};
      ep.e[0] = {EPI_STORE, y2, p, 0, nullptr, nullptr};
      os.attach(ops, P->st);
      gemm_run<T>(p1, ops, ep, os.partial, P->md, P->d_obs, done, P->st);
      // u = v1 - D c1 by FFT or through the band
      d_offpath(P, o1, EPI_SUB_FROM, u, nullptr, v1, nullptr, nullptr, done);
      GemmOpsT<T> ops2{};
      EpisT<T> ep2{};
      ops2.nops = 1;
      ops2.ndig = P->pdig;
      ops2.op[0] = {os.WR, p, y2, p, p, p, N + 1, TRI_UPPER};
      ep2.e[0] = {EPI_STORE, o2, p, 0, nullptr, nullptr};
      os.attach(ops2, P->st);
      gemm_run<T>(p2, ops2, ep2, os.partial, P->md, P->d_obs, done, P->st);
      lhat_sweep<T>(P->md, k, u, o3, false, ident, done, P->st);
      return;
    }
  }
  GemmOpsT<T> ops{};
  EpisT<T> ep{};
  ops.nops = 3;
  ops.ndig = P->pdig;
  ops.op[0] = {os.WRt, p, v2, p, p, p, N + 1, TRI_LOWER};
  ops.op[1] = {os.B, s, o1, s, s, s, 1, TRI_FULL};
  ops.op[2] = {os.Q, s, o1 + s, s, s, s, N, TRI_FULL};
  ep.e[0] = {EPI_STORE, y2, p, 0, nullptr, nullptr};
  ep.e[1] = {EPI_SUB_FROM, u, s, 0, nullptr, v1};
  ep.e[2] = {EPI_SUB_FROM, u + s, s, 0, nullptr, v1 + s};
  os.attach(ops, P->st);
  gemm_run<T>(p1, ops, ep, os.partial, P->md, P->d_obs, done, P->st);
  GemmOpsT<T> ops2{};
  EpisT<T> ep2{};
  ops2.nops = 1;
  ops2.ndig = P->pdig;
  ops2.op[0] = {os.WR, p, y2, p, p, p, N + 1, TRI_UPPER};
  ep2.e[0] = {EPI_STORE, o2, p, 0, nullptr, nullptr};
  os.attach(ops2, P->st);
  gemm_run<T>(p2, ops2, ep2, os.partial, P->md, P->d_obs, done, P->st);
  lhat_sweep<T>(P->md, k, u, o3, false, ident, done, P->st);
}

template <typename T>
static void apply_P(wc4d_problem* P, int which, OpSet<T>& os, const T* v, T* out, const int* done) {
  if (which == WC4D_PRECOND_PD)
    apply_PD<T>(P, os, P->plan_pd1, P->plan_pd2, v, out, done);
  else
    apply_PI<T>(P, os, P->plan_pi1, P->plan_pi2, v, out, done);
}

// ------------------------------------------------------------------ setup
static void copy_in(void* dst, const void* src, size_t bytes, int mem_kind, cudaStream_t st) {
  WC4D_CUDA(cudaMemcpyAsync(dst, src, bytes, mem_kind == WC4D_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                                         : cudaMemcpyHostToDevice, st));
}

static int read_flag(int* d_flag, cudaStream_t st) {
  int h = 0;
  WC4D_CUDA(cudaMemcpyAsync(&h, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  WC4D_CUDA(cudaStreamSynchronize(st));
  return h;
}

// Cholesky + inverse factor of an SPD matrix given in A (overwritten by L).
// The pivot check is read once at the end of setup (a failed factorisation
// only produces non-finite factors meanwhile); each factorisation has its own
// flag slot so the error names the matrix.
static void factor_inverse(wc4d_problem* P, double* A, int m, double* W, double* Wt, double* scratch,
                           const char* what) {
  NvtxRange nvtx_range("wc4d.factor_inverse");
  WC4D_CHECK(P->chol_checks.size() < 12, WC4D_ERR_ARG, "internal: too many factorisations in one setup");
  int* d_info = P->d_flags + 4 + (int)P->chol_checks.size();
  P->chol_checks.push_back({d_info - P->d_flags, what, m});
  cholesky(A, m, d_info, P->st, scratch);
  tri_inverse(A, W, Wt, m, P->st, scratch);
}

// single-op GEMM C = op(At) X with a throwaway plan
static void gemm_once(wc4d_problem* P, const double* At, int64_t lda, const double* X, int64_t ldx, int m, int kdim,
                      int ncols, double* C, int64_t ldc, int mode, int tri = TRI_FULL) {
  GemmPlan plan;
  plan_build(plan, {OpShape{m, kdim, ncols, tri}}, max_gemm_ctas());
  double* partial = nullptr;
  WC4D_CUDA(cudaMalloc(&partial, sizeof(double) * (size_t)std::max(1, plan.nslots) * GEMM_BM * GEMM_BN));
  GemmOps ops{};
  Epis ep{};
  ops.nops = 1;
  ops.op[0] = {At, lda, X, ldx, m, kdim, ncols, tri};
  ep.e[0] = {mode, C, ldc, 0, nullptr, nullptr};
  gemm_run<double>(plan, ops, ep, partial, P->md, P->d_obs, nullptr, P->st);
  WC4D_CUDA(cudaStreamSynchronize(P->st));
  cudaFree(partial);
  plan_free(plan);
}

__global__ void dense_model_kernel(ModelDev md, int t, double* M) {
  const int s = md.s;
  const int64_t total = (int64_t)s * s;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % s), j = (int)(e / s);
    double v = 0.0;
    if (md.kind == WC4D_MODEL_STENCIL3) {
      if (j == (i + s - 1) % s) v += md.c0;
      if (j == i) v += md.c1;
      if (j == (i + 1) % s) v += md.c2;
    } else {
      const int w = md.lo + md.hi + 1;
      int o = j - i;
      if (o > md.hi) o -= s;
      if (o < -md.lo) o += s;
      if (o >= -md.lo && o <= md.hi) v = md.bands[((int64_t)(t - 1) * s + i) * w + o + md.lo];
    }
    M[e] = v;
  }
}

// S[(r0 + i) + (c0 + j) * nS] (+)= alpha * blk[i + j * s] (or its transpose)
__global__ void place_block_kernel(double* S, int nS, int r0, int c0, const double* blk, int s, double alpha,
                                   int accumulate, int transpose) {
  const int64_t total = (int64_t)s * s;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % s), j = (int)(e / s);
    const double v = alpha * (transpose ? blk[j + (int64_t)i * s] : blk[e]);
    double* d = S + (r0 + i) + (int64_t)(c0 + j) * nS;
    *d = accumulate ? *d + v : v;
  }
}

// S[t s + obs[a], t s + obs[b]] += Rinv[a][b] for every time t
__global__ void place_obs_kernel(double* S, int nS, int s, int N, const int* obs, int p, const double* Rinv) {
  const int64_t total = (int64_t)(N + 1) * p * p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e % p), b = (int)((e / p) % p), t = (int)(e / ((int64_t)p * p));
    S[(t * s + obs[a]) + (int64_t)(t * s + obs[b]) * nS] += Rinv[a + (int64_t)b * p];
  }
}

// Exact negative Schur complement S = L^T D^{-1} L + H^T R^{-1} H (Sec. 2.2),
// assembled densely: diagonal blocks D_t^{-1} + M_{t+1}^T D_{t+1}^{-1} M_{t+1}
// + H^T R^{-1} H, off-diagonal blocks -M_{t+1}^T D_{t+1}^{-1} and transpose.
static void build_exact_schur(wc4d_problem* P, double* S, const double* WB, const double* WQ, const double* WR) {
  const int s = P->s, N = P->N, p = P->p, nS = P->nS;
  const int nbk = std::min<int64_t>(((int64_t)nS * nS + 255) / 256, 152 * 16);
  double* Binv = P->alloc<double>((int64_t)s * s);
  double* Qinv = P->alloc<double>((int64_t)s * s);
  double* Rinv = P->alloc<double>((int64_t)p * p);
  double* M = P->alloc<double>((int64_t)s * s);
  double* G = P->alloc<double>((int64_t)s * s);
  double* MG = P->alloc<double>((int64_t)s * s);
  gemm_once(P, WB, s, WB, s, s, s, s, Binv, s, EPI_STORE);   // W^T W = B^{-1}
  gemm_once(P, WQ, s, WQ, s, s, s, s, Qinv, s, EPI_STORE);
  gemm_once(P, WR, p, WR, p, p, p, p, Rinv, p, EPI_STORE);
  launch_fill_d(S, 0.0, (int64_t)nS * nS, P->st);
  for (int t = 0; t <= N; ++t) {
    const double* Dinv = (t == 0) ? Binv : Qinv;
    place_block_kernel<<<nbk, 256, 0, P->st>>>(S, nS, t * s, t * s, Dinv, s, 1.0, 1, 0);
    WC4D_LAUNCH_CHECK();
  }
  for (int t = 1; t <= N; ++t) {
    dense_model_kernel<<<nbk, 256, 0, P->st>>>(P->md, t, M);
    WC4D_LAUNCH_CHECK();
    gemm_once(P, Qinv, s, M, s, s, s, s, G, s, EPI_STORE);   // G = D_t^{-1} M_t
    gemm_once(P, M, s, G, s, s, s, s, MG, s, EPI_STORE);     // M_t^T D_t^{-1} M_t
    place_block_kernel<<<nbk, 256, 0, P->st>>>(S, nS, (t - 1) * s, (t - 1) * s, MG, s, 1.0, 1, 0);
    WC4D_LAUNCH_CHECK();
    place_block_kernel<<<nbk, 256, 0, P->st>>>(S, nS, t * s, (t - 1) * s, G, s, -1.0, 0, 0);
    WC4D_LAUNCH_CHECK();
    place_block_kernel<<<nbk, 256, 0, P->st>>>(S, nS, (t - 1) * s, t * s, G, s, -1.0, 0, 1);
    WC4D_LAUNCH_CHECK();
  }
  place_obs_kernel<<<nbk, 256, 0, P->st>>>(S, nS, s, N, P->d_obs, p, Rinv);
  WC4D_LAUNCH_CHECK();
  launch_symmetrize(S, nS, P->st);
}

static void read_diag_minmax(const double* A, int m, int lim, cudaStream_t st, double& lo, double& hi) {
  std::vector<double> h((size_t)m * m);
  WC4D_CUDA(cudaMemcpyAsync(h.data(), A, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
  WC4D_CUDA(cudaStreamSynchronize(st));
  lo = INFINITY;
  hi = -INFINITY;
  for (int i = 0; i < lim; ++i) {
    lo = std::min(lo, h[(size_t)i * m + i]);
    hi = std::max(hi, h[(size_t)i * m + i]);
  }
}

// R_block (Alg. 3): scaled Frobenius norms of the first super-diagonal channel
// blocks on the device, the cuts on the host, then R zeroed between runs.
static void build_rblock(wc4d_problem* P, double* Rh) {
  const int p = P->p;
  const std::vector<int>& sz = P->rblock_sizes;
  const int pn = (int)sz.size();
  std::vector<double> normvec(pn > 1 ? pn - 1 : 0);
  if (pn > 1) {
    std::vector<int> pst(pn + 1, 0);
    for (int j = 0; j < pn; ++j) pst[j + 1] = pst[j] + sz[j];
    int* d_pst = P->alloc<int>(pn + 1);
    double* d_ss = P->alloc<double>(pn - 1);
    WC4D_CUDA(cudaMemcpyAsync(d_pst, pst.data(), sizeof(int) * (pn + 1), cudaMemcpyHostToDevice, P->st));
    launch_block_sumsq(Rh, p, d_pst, pn - 1, d_ss, P->st);
    WC4D_CUDA(cudaMemcpyAsync(normvec.data(), d_ss, sizeof(double) * (pn - 1), cudaMemcpyDeviceToHost, P->st));
    WC4D_CUDA(cudaStreamSynchronize(P->st));
    for (int j = 0; j + 1 < pn; ++j) normvec[j] = std::sqrt(normvec[j]) / std::sqrt((double)sz[j] * (double)sz[j + 1]);
  }
  const std::vector<int> cuts =
      rblock_cuts(sz, normvec, P->o.rblock_tol, P->o.rblock_maxsize, P->o.rblock_numproc, p);
  P->rhat_param = (double)(cuts.size() + 1);
  if (cuts.empty()) return;
  std::vector<int> run(p);
  for (int i = 0, q = 0; i < p; ++i) {
    while (q < (int)cuts.size() && i >= cuts[q]) ++q;
    run[i] = q;
  }
  int* d_run = P->alloc<int>(p);
  WC4D_CUDA(cudaMemcpyAsync(d_run, run.data(), sizeof(int) * p, cudaMemcpyHostToDevice, P->st));
  launch_zero_across_runs(Rh, p, d_run, P->st);
  WC4D_CUDA(cudaStreamSynchronize(P->st));  // the host label array goes out of scope
}

// Rhat (Sec. 5): copy of R, its diagonal, Alg. 1, Alg. 2 or Alg. 3.
// Rh (p x p) from R (p x p); per-time problems call it once per time level.
static void build_rhat_of(wc4d_problem* P, const double* R, double* Rh, int p, int* d_count) {
  launch_copy_d(Rh, R, (int64_t)p * p, P->st);
  const int rh = P->o.rhat;
  if (rh == WC4D_RHAT_EXACT) return;
  if (rh == WC4D_RHAT_DIAG) {
    launch_keep_diag(Rh, p, P->st);
    return;
  }
  if (rh == WC4D_RHAT_BLOCK) {
    build_rblock(P, Rh);
    return;
  }
  // eigen-decomposition of R by cyclic Jacobi on an even-sized copy; an odd p
  // is padded with one decoupled diagonal entry inside the spectrum (the mean
  // eigenvalue), which neither changes lambda_min/lambda_max nor R_ME's block.
  const int m = (p % 2 == 0) ? p : p + 1;
  double* A = P->alloc<double>((int64_t)m * m);
  double* Vv = P->alloc<double>((int64_t)m * m);
  double* rot = P->alloc<double>((int64_t)2 * m);
  launch_fill_d(A, 0.0, (int64_t)m * m, P->st);
  WC4D_CUDA(cudaMemcpy2DAsync(A, sizeof(double) * m, R, sizeof(double) * p, sizeof(double) * p, p,
                              cudaMemcpyDeviceToDevice, P->st));
  if (m != p) {
    std::vector<double> h((size_t)p * p);
    WC4D_CUDA(cudaMemcpyAsync(h.data(), R, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, P->st));
    WC4D_CUDA(cudaStreamSynchronize(P->st));
    double tr = 0;
    for (int i = 0; i < p; ++i) tr += h[(size_t)i * p + i];
    launch_add_diag(A + (int64_t)p * m + p, 1, m, nullptr, tr / p, P->st);
  }
  jacobi_eigh(A, Vv, m, P->st, rot, d_count, 40);
  double lmin, lmax;
  read_diag_minmax(A, m, p, P->st, lmin, lmax);
  const double kap = P->o.kappa_max;
  if (rh == WC4D_RHAT_RR) {
    // Alg. 1: gamma = (lambda_max - lambda_min kappa_max) / (kappa_max - 1), >= 0
    double gamma = (lmax - lmin * kap) / (kap - 1.0);
    if (gamma < 0.0) gamma = 0.0;
    P->rhat_param = gamma;
    launch_add_diag(Rh, p, p, nullptr, gamma, P->st);
    return;
  }
  // Alg. 2: T = lambda_max / kappa_max; eigenvalues <= T are raised to T
  const double T = lmax / kap;
  P->rhat_param = T;
  if (T <= lmin) return;
  double* U = P->alloc<double>((int64_t)m * m);
  launch_me_scale(A, Vv, m, T, U, nullptr, P->st);
  double* C = P->alloc<double>((int64_t)m * m);
  gemm_once(P, U, m, U, m, m, m, m, C, m, EPI_STORE);  // U^T U = V diag(max(lambda,T)) V^T
  WC4D_CUDA(cudaMemcpy2DAsync(Rh, sizeof(double) * p, C, sizeof(double) * m, sizeof(double) * p, p,
                              cudaMemcpyDeviceToDevice, P->st));
  launch_symmetrize(Rh, p, P->st);
}

static void build_rhat(wc4d_problem* P, int* d_count) {
  NvtxRange nvtx_range("wc4d.build_rhat");
  build_rhat_of(P, P->f64.R, P->d_Rhat, P->p, d_count);
}

static void validate(const wc4d_problem_desc* d, const wc4d_solve_opts* o) {
  WC4D_CHECK(d && o, WC4D_ERR_ARG, "null descriptor or options");
  WC4D_CHECK(d->s >= 2 && d->N >= 0 && d->p >= 1 && (d->p <= d->s || d->p_t != nullptr), WC4D_ERR_ARG,
             "need s >= 2, N >= 0, 1 <= p <= s");
  if (d->p_t != nullptr) {
    int64_t sum = 0;
    for (int t = 0; t <= d->N; ++t) {
      WC4D_CHECK(d->p_t[t] >= 1 && d->p_t[t] <= d->s, WC4D_ERR_ARG, "per-time counts p_t must lie in [1, s]");
      sum += d->p_t[t];
    }
    WC4D_CHECK(sum == d->p, WC4D_ERR_ARG, "per-time counts p_t must sum to p");
    WC4D_CHECK(o != nullptr && (o->rhat == WC4D_RHAT_EXACT || o->rhat == WC4D_RHAT_DIAG ||
                                o->rhat == WC4D_RHAT_RR || o->rhat == WC4D_RHAT_ME),
               WC4D_ERR_ARG, "per-time observation sets take rhat EXACT, DIAG, RR or ME");
    WC4D_CHECK(o->shat == WC4D_SHAT_PAPER, WC4D_ERR_ARG, "per-time observation sets take shat PAPER");
    WC4D_CHECK(o->precision == WC4D_PREC_FP64 || o->precision == WC4D_PREC_DF32 || o->precision == WC4D_PREC_OZAKI,
               WC4D_ERR_ARG, "per-time observation sets run with precision FP64, DF32 or OZAKI");
  }
  WC4D_CHECK(d->mem_kind == WC4D_MEM_HOST || d->mem_kind == WC4D_MEM_DEVICE, WC4D_ERR_ARG, "bad mem_kind");
  WC4D_CHECK(d->obs_idx != nullptr, WC4D_ERR_ARG, "obs_idx is null");
  WC4D_CHECK(d->model_kind == WC4D_MODEL_STENCIL3 || d->model_kind == WC4D_MODEL_BANDED, WC4D_ERR_ARG,
             "bad model_kind");
  if (d->model_kind == WC4D_MODEL_BANDED) {
    WC4D_CHECK(d->band_lo >= 0 && d->band_hi >= 0 && d->band_lo + d->band_hi + 1 <= d->s, WC4D_ERR_ARG,
               "band offsets must satisfy lo, hi >= 0 and lo + hi + 1 <= s");
  }
  WC4D_CHECK(d->cov_kind == WC4D_COV_DENSE || d->cov_kind == WC4D_COV_SOAR || d->cov_kind == WC4D_COV_MSOAR,
             WC4D_ERR_ARG, "bad cov_kind");
  if (d->cov_kind == WC4D_COV_DENSE) {
    WC4D_CHECK(d->B && d->Q && d->R, WC4D_ERR_ARG, "dense covariances missing");
  } else if (d->cov_kind == WC4D_COV_MSOAR) {
    for (const double* m : {d->msoar_b, d->msoar_q})
      WC4D_CHECK(m[0] > 0 && m[1] > 0 && m[2] >= 1 && m[2] == std::floor(m[2]) && 2 * m[2] + 1 <= d->s &&
                     m[2] <= 2048,
                 WC4D_ERR_ARG, "modified SOAR needs amp, L > 0 and an integral maxval, 1 <= maxval <= 2048, "
                               "2 maxval + 1 <= s");
    WC4D_CHECK(d->msoar_psi[0] >= 0 && d->msoar_psi[1] >= 0, WC4D_ERR_ARG, "modified SOAR shifts psi must be >= 0");
    WC4D_CHECK(d->R != nullptr || (d->soar_r[0] > 0 && d->soar_r[1] > 0), WC4D_ERR_ARG,
               "modified SOAR B, Q need a dense R or positive SOAR parameters of R");
    WC4D_CHECK(o->precond == WC4D_PRECOND_PI && o->shat == WC4D_SHAT_PAPER && o->covprod == WC4D_COVPROD_DENSE &&
                   d->p_t == nullptr &&
                   (o->precision == WC4D_PREC_FP64 || o->precision == WC4D_PREC_DF32 ||
                    o->precision == WC4D_PREC_OZAKI),
               WC4D_ERR_ARG,
               "modified SOAR (banded) B, Q run with precond PI, shat PAPER, covprod DENSE, one observation set "
               "and precision FP64, DF32 or OZAKI");
  } else {
    WC4D_CHECK(d->soar_b[1] > 0 && d->soar_q[1] > 0 && d->soar_r[1] > 0 && d->soar_b[0] > 0 && d->soar_q[0] > 0 &&
                   d->soar_r[0] > 0,
               WC4D_ERR_ARG, "SOAR variances and lengths must be positive");
  }
  WC4D_CHECK(o->precond == WC4D_PRECOND_PD || o->precond == WC4D_PRECOND_PI, WC4D_ERR_ARG, "bad precond");
  WC4D_CHECK(o->k >= 1 && o->k <= d->N + 1, WC4D_ERR_ARG, "k must lie in [1, N+1]");
  WC4D_CHECK(o->rhat >= WC4D_RHAT_EXACT && o->rhat <= WC4D_RHAT_BLOCK, WC4D_ERR_ARG, "bad rhat");
  WC4D_CHECK(o->rhat == WC4D_RHAT_EXACT || o->rhat == WC4D_RHAT_DIAG || o->rhat == WC4D_RHAT_BLOCK ||
                 o->kappa_max > 1.0,
             WC4D_ERR_ARG, "kappa_max must exceed 1");
  if (o->rhat == WC4D_RHAT_BLOCK) {
    WC4D_CHECK(o->rblock_count >= 1 && o->rblock_count <= d->p && o->rblock_sizes != nullptr, WC4D_ERR_ARG,
               "RHAT_BLOCK needs 1 <= rblock_count <= p channel block sizes");
    int64_t sum = 0;
    for (int j = 0; j < o->rblock_count; ++j) {
      WC4D_CHECK(o->rblock_sizes[j] >= 1, WC4D_ERR_ARG, "channel block sizes must be >= 1");
      sum += o->rblock_sizes[j];
    }
    WC4D_CHECK(sum == d->p, WC4D_ERR_ARG, "channel block sizes must sum to p");
    WC4D_CHECK(o->rblock_tol >= 0.0 && o->rblock_maxsize >= 0 && o->rblock_numproc >= 0, WC4D_ERR_ARG,
               "need rblock_tol >= 0, rblock_maxsize >= 0, rblock_numproc >= 0");
  }
  WC4D_CHECK(o->lhat == WC4D_LHAT_LM || o->lhat == WC4D_LHAT_I, WC4D_ERR_ARG, "bad lhat");
  WC4D_CHECK(o->shat == WC4D_SHAT_PAPER || o->shat == WC4D_SHAT_EXACT || o->shat == WC4D_SHAT_LEARNED, WC4D_ERR_ARG,
             "bad shat");
  WC4D_CHECK(o->shat != WC4D_SHAT_LEARNED ||
                 (o->precond == WC4D_PRECOND_PD && o->krylov == WC4D_KRYLOV_GMRES && d->N + 1 <= 64),
             WC4D_ERR_ARG, "the learned Schur block needs precond = PD, krylov = GMRES (flexible) and N + 1 <= 64");
  WC4D_CHECK(o->shat != WC4D_SHAT_EXACT || (int64_t)d->s * (d->N + 1) <= 8192, WC4D_ERR_ARG,
             "exact Schur complement limited to s(N+1) <= 8192");
  WC4D_CHECK(o->dhat == WC4D_DHAT_EXACT || o->dhat == WC4D_DHAT_SHIFT, WC4D_ERR_ARG, "bad dhat");
  WC4D_CHECK(o->krylov >= WC4D_KRYLOV_MINRES && o->krylov <= WC4D_KRYLOV_FGMRES, WC4D_ERR_ARG, "bad krylov");
  WC4D_CHECK(!(o->krylov == WC4D_KRYLOV_MINRES && o->precond != WC4D_PRECOND_PD), WC4D_ERR_ARG,
             "MINRES needs the SPD block-diagonal preconditioner P_D");
  WC4D_CHECK(o->tol > 0 && o->maxit >= 1 && o->maxit <= 100000, WC4D_ERR_ARG, "need tol > 0, 1 <= maxit <= 1e5");
  WC4D_CHECK(o->krylov == WC4D_KRYLOV_MINRES || o->maxit <= 2000, WC4D_ERR_ARG,
             "GMRES/FGMRES without restarts keep maxit <= 2000 (Hessenberg column in shared memory)");
  WC4D_CHECK(o->precision == WC4D_PREC_FP64 || o->precision == WC4D_PREC_MIXED || o->precision == WC4D_PREC_DF32 ||
                 o->precision == WC4D_PREC_DF32_P32 || o->precision == WC4D_PREC_OZAKI,
             WC4D_ERR_ARG, "bad precision");
  WC4D_CHECK(o->precision != WC4D_PREC_DF32_P32 || o->krylov == WC4D_KRYLOV_GMRES, WC4D_ERR_ARG,
             "the FP32-preconditioner mode runs the (flexible) DF32 GMRES");
  WC4D_CHECK((o->precision == WC4D_PREC_MIXED) == (o->krylov == WC4D_KRYLOV_FGMRES), WC4D_ERR_ARG,
             "the mixed-precision mode is FGMRES (flexible outer FP64 iteration around an FP32 inner solve), "
             "and FGMRES is only used by it");
  WC4D_CHECK(o->precision != WC4D_PREC_MIXED || (o->inner_iters >= 1 && o->inner_iters <= 200), WC4D_ERR_ARG,
             "inner_iters must lie in [1, 200]");
  WC4D_CHECK(o->covprod == WC4D_COVPROD_DENSE || o->covprod == WC4D_COVPROD_FFT, WC4D_ERR_ARG, "bad covprod");
  WC4D_CHECK(o->prec_digits >= 0 && o->prec_digits <= 7, WC4D_ERR_ARG, "prec_digits must lie in [0, 7]");
  WC4D_CHECK(o->rinv_explicit == 0 || o->rinv_explicit == 1, WC4D_ERR_ARG, "rinv_explicit must be 0 or 1");
  WC4D_CHECK(o->basis_bytes == 0 || o->basis_bytes == 6 || o->basis_bytes == 8, WC4D_ERR_ARG,
             "basis_bytes must be 0, 6 or 8");
  WC4D_CHECK(o->basis_bytes != 6 || (o->krylov == WC4D_KRYLOV_GMRES &&
                                     (o->precision == WC4D_PREC_DF32 || o->precision == WC4D_PREC_DF32_P32 ||
                                      o->precision == WC4D_PREC_OZAKI)),
             WC4D_ERR_ARG, "basis_bytes 6 needs GMRES with precision DF32, DF32_P32 or OZAKI");
  WC4D_CHECK(o->basis_bytes != 6 || o->tol >= 1e-7, WC4D_ERR_ARG,
             "basis_bytes 6 bounds the true residual near 1e-9: needs tol >= 1e-7");
  WC4D_CHECK(o->toeplitz_gemv == WC4D_TOEPLITZ_AUTO || o->toeplitz_gemv == WC4D_TOEPLITZ_OFF, WC4D_ERR_ARG,
             "toeplitz_gemv must be WC4D_TOEPLITZ_AUTO (0) or WC4D_TOEPLITZ_OFF (1)");
  WC4D_CHECK(!o->rinv_explicit || (d->p_t == nullptr && o->precision != WC4D_PREC_MIXED &&
                                   o->precision != WC4D_PREC_DF32_P32 && o->shat != WC4D_SHAT_EXACT),
             WC4D_ERR_ARG,
             "rinv_explicit needs one observation set, precision FP64, DF32 or OZAKI and shat PAPER or LEARNED");
  WC4D_CHECK(o->prec_digits == 0 || o->prec_digits == 7 ||
                 (o->precision == WC4D_PREC_OZAKI && o->krylov == WC4D_KRYLOV_GMRES),
             WC4D_ERR_ARG,
             "reduced-digit preconditioner products need precision OZAKI and the flexible (DF32-basis) GMRES");
  if (o->covprod == WC4D_COVPROD_FFT) {
    WC4D_CHECK(circ_size_ok(d->s), WC4D_ERR_ARG, "covprod FFT needs s a power of two in [64, 8192]");
    WC4D_CHECK(o->precision == WC4D_PREC_FP64 || o->precision == WC4D_PREC_DF32 ||
                   o->precision == WC4D_PREC_OZAKI,
               WC4D_ERR_ARG, "covprod FFT runs with precision FP64, DF32 or OZAKI");
    WC4D_CHECK(o->shat != WC4D_SHAT_EXACT, WC4D_ERR_ARG,
               "covprod FFT does not assemble the exact Schur complement (shat PAPER or LEARNED)");
  }
}

static void setup(wc4d_problem* P, const wc4d_problem_desc* d, const wc4d_solve_opts* o) {
  NvtxRange nvtx_range("wc4d.setup");
  validate(d, o);
  P->o = *o;
  if (o->rhat == WC4D_RHAT_BLOCK) P->rblock_sizes.assign(o->rblock_sizes, o->rblock_sizes + o->rblock_count);
  P->o.rblock_sizes = nullptr;  // caller-owned: read during setup only
  if (P->o.check_every <= 0) P->o.check_every = 4;
  // each outer step of the mixed mode is a whole inner solve: poll every step
  if (o->precision == WC4D_PREC_MIXED) P->o.check_every = 1;
  const int s = d->s, N = d->N, p = d->p;
  P->s = s;
  P->N = N;
  P->p = p;
  P->pertime = (d->p_t != nullptr);
  P->rinv = (o->rinv_explicit != 0);
  P->pdig = (o->precision == WC4D_PREC_OZAKI && o->prec_digits >= 1 && o->prec_digits <= 7) ? o->prec_digits : 7;
  P->ns = (int64_t)(N + 1) * s;
  P->np = P->pertime ? (int64_t)p : (int64_t)(N + 1) * p;  // per-time: p = sum of p_t
  P->n = 2 * P->ns + P->np;
  cudaStream_t st = P->st;
  // flag slots: 0 observation indices, 1 non-finite inputs, 2 R reconditioning,
  // 3 circulant check, 4..15 one per Cholesky factorisation, 16 the tensor-core
  // kernel's give-up code, 17 / 18 the Toeplitz checks of B / Q, 19 that of
  // Q's digit tiles (the setup slots are read once at the end of setup)
  int* d_flag = P->alloc<int>(SETUP_FLAGS);
  P->d_flags = d_flag;
  P->d_kerr = d_flag + 16;
  WC4D_CUDA(cudaMemsetAsync(d_flag, 0, sizeof(int) * SETUP_FLAGS, st));
  // observation operator (the inverse map indexes by obs_idx: checked before it runs)
  P->d_obs = P->alloc<int>(p);
  P->d_inv = P->alloc<int>(P->pertime ? (int64_t)(N + 1) * s : s);
  int pmax = p;  // largest R block
  if (P->pertime) {
    // layout of the per-time nu blocks, R_i blocks and kernel tasks
    P->pt.assign(d->p_t, d->p_t + N + 1);
    std::vector<int> nuoff(N + 2, 0), taskoff(N + 2, 0);
    std::vector<int64_t> aoff(N + 1, 0);
    int64_t el = 0;
    pmax = 0;
    for (int t = 0; t <= N; ++t) {
      const int pi = P->pt[t];
      pmax = std::max(pmax, pi);
      nuoff[t + 1] = nuoff[t] + pi;
      taskoff[t + 1] = taskoff[t] + (pi + PT_ROWS - 1) / PT_ROWS;
      aoff[t] = el;
      el += (int64_t)pi * pi;
    }
    P->pt_elems = el;
    int* d_pt = P->alloc<int>(N + 1);
    int* d_nuoff = P->alloc<int>(N + 2);
    int* d_taskoff = P->alloc<int>(N + 2);
    int64_t* d_aoff = P->alloc<int64_t>(N + 1);
    WC4D_CUDA(cudaMemcpyAsync(d_pt, P->pt.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice, st));
    WC4D_CUDA(cudaMemcpyAsync(d_nuoff, nuoff.data(), sizeof(int) * (N + 2), cudaMemcpyHostToDevice, st));
    WC4D_CUDA(cudaMemcpyAsync(d_taskoff, taskoff.data(), sizeof(int) * (N + 2), cudaMemcpyHostToDevice, st));
    WC4D_CUDA(cudaMemcpyAsync(d_aoff, aoff.data(), sizeof(int64_t) * (N + 1), cudaMemcpyHostToDevice, st));
    P->ptl = PtLayout{N + 1, s, d_pt, d_nuoff, d_aoff, d_taskoff, P->d_obs, taskoff[N + 1]};
    copy_in(P->d_obs, d->obs_idx, sizeof(int) * p, d->mem_kind, st);
    for (int t = 0; t <= N; ++t) {
      const int o0 = nuoff[t], pi = P->pt[t];
      if (d->mem_kind == WC4D_MEM_HOST) {
        for (int r = 0; r < pi; ++r)
          WC4D_CHECK(d->obs_idx[o0 + r] >= 0 && d->obs_idx[o0 + r] < s &&
                         (r == 0 || d->obs_idx[o0 + r] > d->obs_idx[o0 + r - 1]),
                     WC4D_ERR_ARG, "each per-time set of obs_idx must be strictly increasing in [0, s)");
      } else {
        launch_check_obs(P->d_obs + o0, pi, s, d_flag, st);
      }
    }
    WC4D_CHECK(read_flag(d_flag, st) == 0, WC4D_ERR_ARG,
               "each per-time set of obs_idx must be strictly increasing in [0, s)");
    for (int t = 0; t <= N; ++t) launch_inv_map(P->d_obs + nuoff[t], P->pt[t], P->d_inv + (int64_t)t * s, s, st);
    WC4D_CUDA(cudaStreamSynchronize(st));  // the host layout arrays go out of scope
  } else if (d->mem_kind == WC4D_MEM_HOST) {
    for (int r = 0; r < p; ++r)
      WC4D_CHECK(d->obs_idx[r] >= 0 && d->obs_idx[r] < s && (r == 0 || d->obs_idx[r] > d->obs_idx[r - 1]),
                 WC4D_ERR_ARG, "obs_idx must be strictly increasing in [0, s)");
    copy_in(P->d_obs, d->obs_idx, sizeof(int) * p, d->mem_kind, st);
  } else {
    copy_in(P->d_obs, d->obs_idx, sizeof(int) * p, d->mem_kind, st);
    launch_check_obs(P->d_obs, p, s, d_flag, st);
    WC4D_CHECK(read_flag(d_flag, st) == 0, WC4D_ERR_ARG, "obs_idx must be strictly increasing in [0, s)");
  }
  if (!P->pertime) launch_inv_map(P->d_obs, p, P->d_inv, s, st);
  // model
  P->md.kind = d->model_kind;
  P->md.s = s;
  P->md.N = N;
  P->md.c0 = d->stencil[0];
  P->md.c1 = d->stencil[1];
  P->md.c2 = d->stencil[2];
  if (d->model_kind == WC4D_MODEL_BANDED) {
    const int w = d->band_lo + d->band_hi + 1;
    P->d_bands = P->alloc<double>((int64_t)N * s * w);
    if (N > 0 && d->bands) copy_in(P->d_bands, d->bands, sizeof(double) * (size_t)N * s * w, d->mem_kind, st);
    if (N > 0 && !d->bands) WC4D_CUDA(cudaMemsetAsync(P->d_bands, 0, sizeof(double) * (size_t)N * s * w, st));
    P->md.bands = P->d_bands;
    P->md.lo = d->band_lo;
    P->md.hi = d->band_hi;
    launch_check_finite(P->d_bands, (int64_t)N * s * w, d_flag + 1, st);
  }
  // covariances
  OpSet<double>& f = P->f64;
  P->band = (d->cov_kind == WC4D_COV_MSOAR);
  if (P->band) {
    // banded circulant B, Q: the taps of the modified SOAR row (Sec. 6.1) and
    // the diagonal shift |lambda_min| + psi when the circulant is indefinite
    double* d_lmin = P->alloc<double>(2);
    auto taps = [&](const double* m, int& mv) {
      mv = (int)m[2];
      std::vector<double> row(2 * mv + 1);
      const double theta = M_PI / mv;
      for (int i = -mv; i <= mv; ++i) {
        const double dist = 2.0 * std::fabs(std::sin(i * theta / 2.0));
        const double q = dist / m[1];
        row[i + mv] = m[0] * (1.0 + q) * std::exp(-q);
      }
      double* dv = P->alloc<double>(2 * mv + 1);
      WC4D_CUDA(cudaMemcpyAsync(dv, row.data(), sizeof(double) * row.size(), cudaMemcpyHostToDevice, st));
      WC4D_CUDA(cudaStreamSynchronize(st));  // the host row goes out of scope
      return dv;
    };
    P->bandB = taps(d->msoar_b, P->mvB);
    P->bandQ = taps(d->msoar_q, P->mvQ);
    launch_band_lambda_min(P->bandB, P->mvB, s, d_lmin, st);
    launch_band_lambda_min(P->bandQ, P->mvQ, s, d_lmin + 1, st);
    double lmin[2];
    WC4D_CUDA(cudaMemcpyAsync(lmin, d_lmin, sizeof lmin, cudaMemcpyDeviceToHost, st));
    WC4D_CUDA(cudaStreamSynchronize(st));
    P->deltaB = lmin[0] < 0.0 ? std::fabs(lmin[0]) + d->msoar_psi[0] : 0.0;
    P->deltaQ = lmin[1] < 0.0 ? std::fabs(lmin[1]) + d->msoar_psi[1] : 0.0;
    WC4D_CHECK(lmin[0] + P->deltaB > 0.0 && lmin[1] + P->deltaQ > 0.0, WC4D_ERR_NOT_SPD,
               "modified SOAR B or Q is singular (lambda_min + shift = 0)");
  } else {
    f.B = P->alloc<double>((int64_t)s * s);
    f.Q = P->alloc<double>((int64_t)s * s);
  }
  // R: one p x p matrix, or the per-time blocks R_0..R_N one after another
  double* Rdst = nullptr;
  int64_t Rcnt = 0;
  if (P->pertime) {
    P->ptR = P->alloc<double>(P->pt_elems);
    Rdst = P->ptR;
    Rcnt = P->pt_elems;
  } else {
    f.R = P->alloc<double>((int64_t)p * p);
    Rdst = f.R;
    Rcnt = (int64_t)p * p;
  }
  if (d->cov_kind == WC4D_COV_DENSE || (P->band && d->R != nullptr)) {
    if (!P->band) {
      copy_in(f.B, d->B, sizeof(double) * (size_t)s * s, d->mem_kind, st);
      copy_in(f.Q, d->Q, sizeof(double) * (size_t)s * s, d->mem_kind, st);
    }
    copy_in(Rdst, d->R, sizeof(double) * (size_t)Rcnt, d->mem_kind, st);
  } else {
    double* tab = P->alloc<double>(s);
    if (!P->band) {
      launch_soar_fill(f.B, s, nullptr, s, d->soar_b[0], d->soar_b[1], tab, st);
      launch_soar_fill(f.Q, s, nullptr, s, d->soar_q[0], d->soar_q[1], tab, st);
    }
    if (P->pertime) {
      for (int t = 0, o0 = 0; t <= N; o0 += P->pt[t], ++t) {
        int64_t a0 = 0;
        for (int u = 0; u < t; ++u) a0 += (int64_t)P->pt[u] * P->pt[u];
        launch_soar_fill(P->ptR + a0, P->pt[t], P->d_obs + o0, s, d->soar_r[0], d->soar_r[1], tab, st);
      }
    } else {
      launch_soar_fill(f.R, p, P->d_obs, s, d->soar_r[0], d->soar_r[1], tab, st);
    }
  }
  if (!P->band) {
    launch_check_finite(f.B, (int64_t)s * s, d_flag + 1, st);
    launch_check_finite(f.Q, (int64_t)s * s, d_flag + 1, st);
  }
  launch_check_finite(Rdst, Rcnt, d_flag + 1, st);
  // circulant B and Q (WC4D_COVPROD_FFT): twiddles and spectra
  P->circ = (o->covprod == WC4D_COVPROD_FFT);
  if (P->circ) {
    if (d->cov_kind == WC4D_COV_DENSE) {
      // the caller's B and Q must equal the circulants of their first columns
      launch_circ_check(f.B, s, 1e-12, d_flag + 3, st);
      launch_circ_check(f.Q, s, 1e-12, d_flag + 3, st);
      WC4D_CHECK(read_flag(d_flag + 3, st) == 0, WC4D_ERR_ARG,
                 "covprod FFT: B or Q is not circulant (entries differ from the circulant of the first column by "
                 "more than 1e-12 of the diagonal)");
    }
    P->tw = P->alloc<double2>(s);
    launch_circ_twiddles(P->tw, s, st);
    auto spectrum = [&](const double* M, double shift, int invert, const char* what) {
      WC4D_CHECK(P->chol_checks.size() < 12, WC4D_ERR_ARG, "internal: too many setup checks");
      int* slot = P->d_flags + 4 + (int)P->chol_checks.size();
      P->chol_checks.push_back({slot - P->d_flags, what, s, true});
      double* lam = P->alloc<double>(s);
      launch_circ_spectrum(M, s, P->tw, shift, invert, lam, slot, st);
      return lam;
    };
    P->lamB = spectrum(f.B, 0.0, 0, "B");
    P->lamQ = spectrum(f.Q, 0.0, 0, "Q");
    if (o->precond == WC4D_PRECOND_PD) {
      const double delta = (o->dhat == WC4D_DHAT_SHIFT) ? o->dhat_delta : 0.0;
      P->lamBi = spectrum(f.B, delta, 1, "Bhat");
      P->lamQi = spectrum(f.Q, delta, 1, "Qhat");
    }
    P->circ_df = (o->precision != WC4D_PREC_FP64);
    if (P->circ_df) {
      auto split = [&](const double* l) {
        if (!l) return (float2*)nullptr;
        float2* dv = P->alloc<float2>(s);
        launch_circ_split(l, dv, s, st);
        return dv;
      };
      P->twdf = P->alloc<float4>(s);
      launch_circ_split(reinterpret_cast<const double*>(P->tw), reinterpret_cast<float2*>(P->twdf), 2 * s, st);
      P->lamBdf = split(P->lamB);
      P->lamQdf = split(P->lamQ);
      P->lamBidf = split(P->lamBi);
      P->lamQidf = split(P->lamQi);
    }
  }
  const int mmax = std::max(s, pmax);
  double* scratch = P->alloc<double>((int64_t)mmax * 64 + 64 * 64 * 2);
  // factorisation workspace: s x s only where B and Q are factored (dense P_D)
  const bool factor_d = (o->precond == WC4D_PRECOND_PD) && !P->circ && !P->band;
  const int wdim = factor_d ? mmax : pmax;
  double* work = P->alloc<double>((int64_t)wdim * wdim);
  if (P->pertime) {
    // Rhat_i from each R_i alone (Sec. 5), then W_i = chol(Rhat_i)^-1 and W_i^T;
    // one pivot-check slot for all time levels
    NvtxRange nvtx_r("wc4d.build_rhat");
    P->ptRh = P->alloc<double>(P->pt_elems);
    P->ptW = P->alloc<double>(P->pt_elems);
    P->ptWt = P->alloc<double>(P->pt_elems);
    WC4D_CHECK(P->chol_checks.size() < 12, WC4D_ERR_ARG, "internal: too many setup checks");
    int* slot = P->d_flags + 4 + (int)P->chol_checks.size();
    P->chol_checks.push_back({slot - P->d_flags, "a per-time Rhat_i", pmax});
    double param0 = 0.0;
    int64_t a0 = 0;
    for (int t = 0; t <= N; ++t) {
      const int pi = P->pt[t];
      build_rhat_of(P, P->ptR + a0, P->ptRh + a0, pi, d_flag + 2);
      if (t == 0) param0 = P->rhat_param;
      launch_copy_d(work, P->ptRh + a0, (int64_t)pi * pi, st);
      cholesky(work, pi, slot, st, scratch);
      tri_inverse(work, P->ptW + a0, P->ptWt + a0, pi, st, scratch);
      a0 += (int64_t)pi * pi;
    }
    P->rhat_param = param0;
  } else {
  // Rhat and its inverse factor
  P->d_Rhat = P->alloc<double>((int64_t)p * p);
  build_rhat(P, d_flag + 2);
  f.WR = P->alloc<double>((int64_t)p * p);
  f.WRt = P->alloc<double>((int64_t)p * p);
  launch_copy_d(work, P->d_Rhat, (int64_t)p * p, st);
  factor_inverse(P, work, p, f.WR, f.WRt, scratch, "Rhat");
  if (P->rinv && o->precision == WC4D_PREC_FP64) {
    // Rhat^-1 = W^T W (W = chol(Rhat)^-1 lower: row i of W^T meets k >= i only);
    // the double-float modes form it below from W's split
    f.Rinv = P->alloc<double>((int64_t)p * p);
    gemm_once(P, f.WR, p, f.WR, p, p, p, p, f.Rinv, p, EPI_STORE, TRI_UPPER);
    launch_symmetrize(f.Rinv, p, st);
  }
  }
  // Dhat factors (P_D only)
  P->have_pd = (o->precond == WC4D_PRECOND_PD);
  if (P->have_pd && !P->circ) {
    const double delta = (o->dhat == WC4D_DHAT_SHIFT) ? o->dhat_delta : 0.0;
    f.WB = P->alloc<double>((int64_t)s * s);
    f.WBt = P->alloc<double>((int64_t)s * s);
    f.WQ = P->alloc<double>((int64_t)s * s);
    f.WQt = P->alloc<double>((int64_t)s * s);
    launch_copy_d(work, f.B, (int64_t)s * s, st);
    if (delta != 0.0) launch_add_diag(work, s, s, nullptr, delta, st);
    factor_inverse(P, work, s, f.WB, f.WBt, scratch, "Bhat");
    launch_copy_d(work, f.Q, (int64_t)s * s, st);
    if (delta != 0.0) launch_add_diag(work, s, s, nullptr, delta, st);
    factor_inverse(P, work, s, f.WQ, f.WQt, scratch, "Qhat");
    if (o->shat == WC4D_SHAT_EXACT) {
      // S uses the exact D and R (Sec. 2.2): factors of B, Q, R themselves
      double *eB = f.WB, *eQ = f.WQ, *eR = f.WR;
      if (delta != 0.0 || o->rhat != WC4D_RHAT_EXACT) {
        double* tmpt = P->alloc<double>((int64_t)mmax * mmax);
        eB = P->alloc<double>((int64_t)s * s);
        eQ = P->alloc<double>((int64_t)s * s);
        eR = P->alloc<double>((int64_t)p * p);
        launch_copy_d(work, f.B, (int64_t)s * s, st);
        factor_inverse(P, work, s, eB, tmpt, scratch, "B");
        launch_copy_d(work, f.Q, (int64_t)s * s, st);
        factor_inverse(P, work, s, eQ, tmpt, scratch, "Q");
        launch_copy_d(work, f.R, (int64_t)p * p, st);
        factor_inverse(P, work, p, eR, tmpt, scratch, "R");
      }
      P->nS = s * (N + 1);
      const int nS = P->nS;
      double* S = P->alloc<double>((int64_t)nS * nS);
      build_exact_schur(P, S, eB, eQ, eR);
      f.WS = P->alloc<double>((int64_t)nS * nS);
      f.WSt = P->alloc<double>((int64_t)nS * nS);
      double* sscr = P->alloc<double>((int64_t)nS * 64 + 64 * 64 * 2);
      factor_inverse(P, S, nS, f.WS, f.WSt, sscr, "S");
    }
  }
  // GEMM schedules
  const bool dfm = (o->precision != WC4D_PREC_FP64);
  const bool ozm = (o->precision == WC4D_PREC_OZAKI);
  const int C = ozm ? oz_resident_ctas() : max_gemm_ctas(dfm);
  const int cm = ozm ? COST_TC : (dfm ? COST_DF32 : COST_FP64);
  if (P->pertime && P->circ) {
    // every product is a transform or a per-time product: no GEMM plans
  } else if (P->pertime) {
    // the R family runs in the per-time kernel: plans for the D products only
    plan_build(P->plan_A, {{s, s, 1, TRI_FULL}, {s, s, N, TRI_FULL}}, C, cm);
    if (P->have_pd) {
      plan_build(P->plan_pd1, {{s, s, 1, TRI_LOWER}, {s, s, N, TRI_LOWER}, {s, s, N, TRI_FULL}}, C, cm);
      plan_build(P->plan_pd2, {{s, s, 1, TRI_UPPER}, {s, s, N, TRI_UPPER}, {s, s, 1, TRI_FULL}}, C, cm);
    }
    plan_build(P->plan_pi1, {{s, s, 1, TRI_FULL}, {s, s, N, TRI_FULL}}, C, cm);
  } else if (P->circ || P->band) {
    // only the R family remains on the product path
    plan_build(P->plan_A, {{p, p, N + 1, TRI_FULL}}, C, cm);
    const int t1 = P->rinv ? TRI_FULL : TRI_LOWER;
    if (P->have_pd) {
      plan_build(P->plan_pd1, {{p, p, N + 1, t1}}, C, cm);
      if (!P->rinv) plan_build(P->plan_pd2, {{p, p, N + 1, TRI_UPPER}}, C, cm);
    }
    plan_build(P->plan_pi1, {{p, p, N + 1, t1}}, C, cm);
    if (!P->rinv) plan_build(P->plan_pi2, {{p, p, N + 1, TRI_UPPER}}, C, cm);
  } else if (P->rinv) {
    // Rhat^-1 as one full product, in the first launch of each preconditioner
    plan_build(P->plan_A, {{s, s, 1, TRI_FULL}, {s, s, N, TRI_FULL}, {p, p, N + 1, TRI_FULL}}, C, cm);
    if (P->have_pd) {
      plan_build(P->plan_pd1, {{p, p, N + 1, TRI_FULL}, {s, s, 1, TRI_LOWER}, {s, s, N, TRI_LOWER},
                               {s, s, N, TRI_FULL}}, C, cm);
      plan_build(P->plan_pd2, {{s, s, 1, TRI_UPPER}, {s, s, N, TRI_UPPER}, {s, s, 1, TRI_FULL}}, C, cm);
    }
    plan_build(P->plan_pi1, {{p, p, N + 1, TRI_FULL}, {s, s, 1, TRI_FULL}, {s, s, N, TRI_FULL}}, C, cm);
  } else {
  plan_build(P->plan_A, {{s, s, 1, TRI_FULL}, {s, s, N, TRI_FULL}, {p, p, N + 1, TRI_FULL}}, C, cm);
  if (P->have_pd) {
    if (o->shat == WC4D_SHAT_EXACT) {
      plan_build(P->plan_pd1, {{s, s, 1, TRI_LOWER}, {s, s, N, TRI_LOWER}, {p, p, N + 1, TRI_LOWER},
                               {P->nS, P->nS, 1, TRI_LOWER}}, C, cm);
      plan_build(P->plan_pd2, {{s, s, 1, TRI_UPPER}, {s, s, N, TRI_UPPER}, {p, p, N + 1, TRI_UPPER},
                               {P->nS, P->nS, 1, TRI_UPPER}}, C, cm);
    } else {
      plan_build(P->plan_pd1, {{s, s, 1, TRI_LOWER}, {s, s, N, TRI_LOWER}, {p, p, N + 1, TRI_LOWER},
                               {s, s, N, TRI_FULL}}, C, cm);
      plan_build(P->plan_pd2, {{s, s, 1, TRI_UPPER}, {s, s, N, TRI_UPPER}, {p, p, N + 1, TRI_UPPER},
                               {s, s, 1, TRI_FULL}}, C, cm);
    }
  }
  plan_build(P->plan_pi1, {{p, p, N + 1, TRI_LOWER}, {s, s, 1, TRI_FULL}, {s, s, N, TRI_FULL}}, C, cm);
  plan_build(P->plan_pi2, {{p, p, N + 1, TRI_UPPER}}, C, cm);
  }
  int slots = std::max({P->plan_A.nslots, P->plan_pd1.nslots, P->plan_pd2.nslots, P->plan_pi1.nslots,
                        P->plan_pi2.nslots, 1});
  const GemmPlan* plans[5] = {&P->plan_A, &P->plan_pd1, &P->plan_pd2, &P->plan_pi1, &P->plan_pi2};
  int64_t slot_rows = 0;  // slots x rows per slot over the plans
  for (const GemmPlan* pl : plans) slot_rows = std::max<int64_t>(slot_rows, (int64_t)pl->nslots * pl->bm);
  f.partial = P->alloc<double>(std::max<int64_t>(slot_rows, GEMM_BM) * GEMM_BN);
  f.t1 = P->alloc<double>(P->n);
  f.t2 = P->alloc<double>(P->n);
  f.t3 = P->alloc<double>(P->n);
  if (o->precision != WC4D_PREC_FP64) {
    f.df32 = 1;
    f.xcap = 2 * P->n;
    f.xh = P->alloc<float>(f.xcap);
    f.xl = P->alloc<float>(f.xcap);
    auto add = [&](const double* m, int64_t cnt) {
      if (!m) return;
      float* h = P->alloc<float>(cnt);
      float* l = P->alloc<float>(cnt);
      launch_split_df(m, h, l, cnt, st);
      f.splits.push_back({m, Split{h, l}});
    };
    if (!P->circ && !P->band) {  // circulant B, Q never meet the product kernels
      add(f.B, (int64_t)s * s);
      add(f.Q, (int64_t)s * s);
    }
    add(f.R, (int64_t)p * p);
    add(f.WR, (int64_t)p * p);
    add(f.WRt, (int64_t)p * p);
    if (P->rinv) {
      // Rhat^-1 = W^T W as a double-float product on the FP32 pipe, both
      // operands W's split (X = W with leading dimension p)
      f.Rinv = P->alloc<double>((int64_t)p * p);
      const Split sw = f.split_of(f.WR);
      GemmPlan plan;
      plan_build(plan, {OpShape{p, p, p, TRI_UPPER}}, max_gemm_ctas(true), COST_DF32);
      double* part = P->alloc<double>((int64_t)std::max(1, plan.nslots) * GEMM_BM * GEMM_BN);
      GemmOps ops{};
      Epis ep{};
      ops.nops = 1;
      ops.df32 = 1;
      ops.op[0] = {f.WR, p, f.WR, p, p, p, p, TRI_UPPER};
      ops.op[0].Ah = sw.h;
      ops.op[0].Al = sw.l;
      ops.op[0].Xh = sw.h;
      ops.op[0].Xl = sw.l;
      ep.e[0] = {EPI_STORE, f.Rinv, p, 0, nullptr, nullptr};
      gemm_run<double>(plan, ops, ep, part, P->md, P->d_obs, nullptr, st);
      launch_symmetrize(f.Rinv, p, st);
      add(f.Rinv, (int64_t)p * p);
    }
    add(f.WB, (int64_t)s * s);
    add(f.WBt, (int64_t)s * s);
    add(f.WQ, (int64_t)s * s);
    add(f.WQt, (int64_t)s * s);
    if (f.WS) {
      add(f.WS, (int64_t)P->nS * P->nS);
      add(f.WSt, (int64_t)P->nS * P->nS);
    }
  }
  if (ozm) {
    // digit forms of the operators that meet two or more right-hand sides
    // (the Q family with N >= 2 time levels, the R family with N + 1 >= 2)
    f.tc = 1;
    auto dig = [&](const double* m, int rows) {
      if (!m) return;
      const int64_t rp = (int64_t)(rows + OZ_BM - 1) / OZ_BM * OZ_BM;
      uint16_t* d = P->alloc<uint16_t>(oz_operator_elems(rows, rows));
      float* sc = P->alloc<float>(rp);
      launch_oz_rows(m, rows, rows, rows, d, sc, st);
      f.digits.push_back({m, Digits{d, sc}});
    };
    if (N >= 2 && !P->circ && !P->band) {
      dig(f.Q, s);
      dig(f.WQ, s);
      dig(f.WQt, s);
    }
    if (N + 1 >= 2) {
      dig(f.R, p);
      dig(f.Rinv, p);
      dig(f.WR, p);
      dig(f.WRt, p);
    }
    if (!P->circ && !P->band && o->toeplitz_gemv == WC4D_TOEPLITZ_AUTO) {
      // one-column products of B and Q from their first row when they are
      // symmetric Toeplitz (checked bitwise; registered at the end of setup)
      auto toep = [&](const double* m, int slot) {
        const Split sp = f.split_of(m);
        if (!m || !sp.h) return;
        const int64_t cnt = 4 * oz_toeplitz_stride(s);
        float* th = P->alloc<float>(cnt);
        float* tl = P->alloc<float>(cnt);
        launch_oz_toeplitz(m, s, s, sp.h, sp.l, th, tl, d_flag + slot, st);
        P->toep_checks.push_back({m, Split{th, tl}, slot});
      };
      toep(f.B, 17);
      toep(f.Q, 18);
      // Q's digit tiles (N >= 2): the product kernel reads one tile per
      // offset 128 R - 16 K when every tile equals that one (checked bitwise)
      const Digits dq = f.digits_of(f.Q);
      if (f.Q && dq.d) {
        launch_oz_toeplitz_tiles(dq.d, s, s, d_flag + 19, st);
        P->toep_checks.push_back({f.Q, Split{}, 19});
      }
    }
    int64_t xe = 0, xsc = 0, xgc = 0;
    for (const GemmPlan* pl : plans) {
      int64_t e = 0, c = 0, gg = 0;
      for (int q = 0; q < pl->nops; ++q) {
        e += oz_x_elems(pl->shape[q].kdim, pl->shape[q].ncols);
        c += (int64_t)oz_wide_tiles(pl->shape[q].ncols) * OZ_BN;
        if (oz_gemv_col(pl->shape[q].ncols) >= 0) gg += 2 * ((pl->shape[q].kdim + 3) / 4 * 4);
      }
      xe = std::max(xe, e);
      xsc = std::max(xsc, c);
      xgc = std::max(xgc, gg);
    }
    f.xgcap = std::max<int64_t>(xgc, 4);
    f.xg = P->alloc<float>(f.xgcap);
    f.xdcap = std::max<int64_t>(xe, 8);
    f.xd = P->alloc<uint16_t>(f.xdcap);
    f.xscap = std::max<int64_t>(xsc, 1);
    f.xs = P->alloc<float>(f.xscap);
    f.tc_err = P->d_kerr;
  }
  if (o->precision == WC4D_PREC_MIXED || o->precision == WC4D_PREC_DF32_P32) {
    OpSet<float>& g = P->f32;
    auto to32 = [&](const double* src, int64_t cnt) {
      if (!src) return (float*)nullptr;
      float* d = P->alloc<float>(cnt);
      launch_to_float(src, d, cnt, st);
      return d;
    };
    g.B = to32(f.B, (int64_t)s * s);
    g.Q = to32(f.Q, (int64_t)s * s);
    g.R = to32(f.R, (int64_t)p * p);
    g.WR = to32(f.WR, (int64_t)p * p);
    g.WRt = to32(f.WRt, (int64_t)p * p);
    g.WB = to32(f.WB, (int64_t)s * s);
    g.WBt = to32(f.WBt, (int64_t)s * s);
    g.WQ = to32(f.WQ, (int64_t)s * s);
    g.WQt = to32(f.WQt, (int64_t)s * s);
    if (f.WS) {
      g.WS = to32(f.WS, (int64_t)P->nS * P->nS);
      g.WSt = to32(f.WSt, (int64_t)P->nS * P->nS);
    }
    g.partial = P->alloc<float>((int64_t)slots * GEMM_BM * GEMM_BN);
    g.t1 = P->alloc<float>(P->n);
    g.t2 = P->alloc<float>(P->n);
    g.t3 = P->alloc<float>(P->n);
    P->stage = P->alloc<float>(P->n);
  }
  if (o->precision == WC4D_PREC_DF32_P32) P->zf = P->alloc<float>(P->n);
  if (o->precision == WC4D_PREC_MIXED) {
    const int mi = o->inner_iters;
    P->mi = mi;
    P->Vi = P->alloc<float>((int64_t)(mi + 1) * P->n);
    P->Zi = P->alloc<float>((int64_t)mi * P->n);
    P->Hi = P->alloc<double>((int64_t)(mi + 1) * mi);
    P->csi = P->alloc<double>(mi + 1);
    P->sni = P->alloc<double>(mi + 1);
    P->gi = P->alloc<double>(mi + 2);
    P->yi = P->alloc<double>(mi + 1);
    P->h1i = P->alloc<double>(mi + 2);
    P->h2i = P->alloc<double>(mi + 2);
    P->hnexti = P->alloc<double>(2);
    P->bnormi = P->alloc<double>(2);
    P->parti = P->alloc<double>((int64_t)std::max(DOT_BLOCKS, orth_chunks(P->n)) * (mi + 2));
    P->part2i = P->alloc<double>(DOT_BLOCKS);
    P->stat_in = P->alloc<DevStatus>(1);
  }
  // Krylov workspace
  const int64_t n = P->n;
  P->maxit = o->maxit;
  const int64_t nvec = (o->krylov == WC4D_KRYLOV_MINRES) ? 12 : (int64_t)o->maxit + 1;
  P->split_basis = (o->krylov != WC4D_KRYLOV_MINRES) && (o->precision != WC4D_PREC_FP64);
  P->dcgs = (o->krylov == WC4D_KRYLOV_GMRES) &&
            (o->precision == WC4D_PREC_DF32 || o->precision == WC4D_PREC_DF32_P32 ||
             o->precision == WC4D_PREC_OZAKI);
  P->b6 = P->dcgs && o->basis_bytes == 6;
  if (P->split_basis) {
    // leading dimension padded to 4 floats (16-byte loads); padding stays zero.
    // The 6-byte basis keeps its BF16 low parts in half the low-part array
    // (16-bit words, the same leading dimension in elements).
    P->ldb = (n + 3) / 4 * 4;
    const size_t lo_size = P->b6 ? 2 : sizeof(float);
    P->Vh = P->alloc<float>(nvec * P->ldb);
    P->Vl = P->alloc<float>(P->b6 ? nvec * P->ldb / 2 : nvec * P->ldb);
    P->wh = P->alloc<float>(P->ldb);
    P->wl = P->alloc<float>(P->ldb);
    if (P->ldb != n) {  // only the padding of each basis vector must read zero
      const size_t pitch = sizeof(float) * P->ldb, width = sizeof(float) * (P->ldb - n);
      WC4D_CUDA(cudaMemset2DAsync(P->Vh + n, pitch, 0, width, nvec, st));
      WC4D_CUDA(cudaMemset2DAsync(reinterpret_cast<char*>(P->Vl) + lo_size * n, lo_size * P->ldb, 0,
                                  lo_size * (P->ldb - n), nvec, st));
    }
    WC4D_CUDA(cudaMemsetAsync(P->wh, 0, sizeof(float) * P->ldb, st));
    WC4D_CUDA(cudaMemsetAsync(P->wl, 0, sizeof(float) * P->ldb, st));
    P->vcur = P->alloc<double>(n);
    P->wbuf = P->alloc<double>(n);
    P->V = P->alloc<double>(n);  // r0 staging only
  } else {
    P->V = P->alloc<double>(nvec * n);
  }
  if (o->krylov != WC4D_KRYLOV_MINRES) P->Z = P->alloc<double>((int64_t)(o->maxit + (P->dcgs ? 1 : 0)) * n);
  const int ldh = o->maxit + 1;
  P->H = P->alloc<double>((int64_t)ldh * o->maxit);
  if (P->dcgs) {
    P->Hraw = P->alloc<double>((int64_t)ldh * o->maxit);
    P->Tm = P->alloc<double>((int64_t)ldh * (o->maxit + 1));
    P->dcst = P->alloc<double>(DC_COUNT);
    P->bprev = P->alloc<double>(o->maxit + 2);
    P->cprev = P->alloc<double>(o->maxit + 2);
    P->ecoef = P->alloc<double>(o->maxit + 2);
    P->red = P->alloc<double>(2 * (int64_t)o->maxit + 4);
    P->yhat = P->alloc<double>(o->maxit + 1);
    P->hcbuf = P->alloc<double>(o->maxit + 2);
  }
  P->cs = P->alloc<double>(o->maxit + 1);
  P->sn = P->alloc<double>(o->maxit + 1);
  P->g = P->alloc<double>(o->maxit + 2);
  P->y = P->alloc<double>(o->maxit + 1);
  P->h1 = P->alloc<double>(o->maxit + 2);
  P->h2 = P->alloc<double>(o->maxit + 2);
  P->hnext = P->alloc<double>(2);
  P->bnorm = P->alloc<double>(2);
  P->scal = P->alloc<double>(8);
  P->part = P->alloc<double>((int64_t)std::max(DOT_BLOCKS, orth_chunks(P->n)) * (2 * (int64_t)o->maxit + 4));
  P->part2 = P->alloc<double>(DOT_BLOCKS);
  P->part3 = P->alloc<double>(DOT_BLOCKS);
  P->sc = P->alloc<double>(2 * MS_COUNT);
  P->rhs = P->alloc<double>(n);
  P->x = P->alloc<double>(n);
  P->r = P->alloc<double>(n);
  P->x0 = P->alloc<double>(n);
  P->stat = P->alloc<DevStatus>(1);
  if (o->shat == WC4D_SHAT_LEARNED) {
    const int64_t len = (int64_t)(N + 1) * s;
    P->net_in = P->alloc<float>(len);
    P->net_out = P->alloc<float>(len);
    for (int l = 0; l < 3; ++l) P->net_act[l] = P->alloc<float>(64 * (int64_t)s);
    P->net_nrm2 = P->alloc<double>(1);
    P->net_part = P->alloc<double>(DOT_BLOCKS);
    P->net_params = P->alloc<float>(NetShape{N + 1, 64, s}.nparams());
  }
  P->h_stat = (DevStatus*)pinned_get();
  P->h_scal = (double*)pinned_get();
  // the deferred checks: non-finite inputs, then each factorisation's pivots
  int* hf = (int*)pinned_get();
  WC4D_CUDA(cudaMemcpyAsync(hf, d_flag, sizeof(int) * SETUP_FLAGS, cudaMemcpyDeviceToHost, st));
  WC4D_CUDA(cudaStreamSynchronize(st));
  int hflags[SETUP_FLAGS];
  std::memcpy(hflags, hf, sizeof hflags);
  pinned_put(hf);
  WC4D_CHECK(hflags[1] == 0, WC4D_ERR_NONFINITE, "non-finite entries in the model or covariance inputs");
  for (const auto& ck : P->chol_checks) {
    if (hflags[ck.slot] != 0 && ck.spectrum) {
      char buf[160];
      snprintf(buf, sizeof buf, "circulant %s is not SPD: a spectrum value (plus the shift) is not positive", ck.what);
      throw Error{WC4D_ERR_NOT_SPD, buf};
    }
    if (hflags[ck.slot] != 0) {
      char buf[160];
      snprintf(buf, sizeof buf, "Cholesky of %s failed: non-positive pivot %d of %d", ck.what, hflags[ck.slot], ck.m);
      throw Error{WC4D_ERR_NOT_SPD, buf};
    }
  }
  for (const auto& tc : P->toep_checks) {
    if (hflags[tc.slot] != 0) continue;
    if (tc.rows.h)
      P->f64.toeps.push_back({tc.op, tc.rows});
    else
      P->f64.toep_tiled.push_back(tc.op);
  }
}

// ------------------------------------------------------------------ solves
static void fetch_stat(wc4d_problem* P) {
  WC4D_CUDA(cudaMemcpyAsync(P->h_stat, P->stat, sizeof(DevStatus), cudaMemcpyDeviceToHost, P->st));
  WC4D_CUDA(cudaStreamSynchronize(P->st));
}

// ||rhs - A x|| / ||rhs|| in FP64, read back to the host
static double true_relres(wc4d_problem* P, const double* rhs, const double* x) {
  NvtxRange nvtx_range("wc4d.true_residual");
  apply_A<double>(P, P->f64, P->plan_A, x, P->r, nullptr);
  vec_sub(rhs, P->r, P->r, P->n, P->st);
  dot_partial<double>(P->r, P->r, P->n, P->part3, nullptr, P->st);
  dot_finish(P->part3, P->scal + 1, 1, P->st);
  WC4D_CUDA(cudaMemcpyAsync(P->h_scal, P->scal, sizeof(double) * 2, cudaMemcpyDeviceToHost, P->st));
  WC4D_CUDA(cudaStreamSynchronize(P->st));
  const double bn = P->h_scal[0];
  return P->h_scal[1] / (bn > 0 ? bn : 1.0);
}

static void resume_after_false_stop(wc4d_problem* P, double est, double relres) {
  P->h_stat->done = 0;
  P->h_stat->tol_est = est * (P->o.tol / relres) * 0.5;
  WC4D_CUDA(cudaMemcpyAsync(P->stat, P->h_stat, sizeof(DevStatus), cudaMemcpyHostToDevice, P->st));
  WC4D_CUDA(cudaStreamSynchronize(P->st));
}

// The tensor-core product kernel sets the problem's error word when one of
// its bounded waits gives up; every output of that launch (and of what was
// computed from it) is then invalid.  Reads and clears the word (the stream
// must be synchronised) and reports WC4D_ERR_TIMEOUT.
static void check_kernel_waits(wc4d_problem* P) {
  if (!P->d_kerr) return;
  int e = 0;
  WC4D_CUDA(cudaMemcpy(&e, P->d_kerr, sizeof(int), cudaMemcpyDeviceToHost));
  if (e == 0) return;
  WC4D_CUDA(cudaMemset(P->d_kerr, 0, sizeof(int)));
  throw Error{WC4D_ERR_TIMEOUT, "tensor-core product kernel: a bounded wait gave up (role " + std::to_string(e) +
                                    "); the outputs of that launch are invalid"};
}

// Per-component product counts in the convention of Tables 4 and 5: one count
// per time block touched, from the number of A and P applies of the solve.
// A v: N+1 R_i and N+1 D_i products, 2N model products (L and L^T).  P_D^{-1}:
// N+1 Dhat_i^{-1} and N+1 Rhat_i^{-1} applies, N+1 D_i products and
// 2(N - floor(N/k)) model products in the two Lhat sweeps (paper Shat; none
// for the exact S or for Lhat = L_I).  P_I^{-1}: N+1 Rhat_i^{-1}, N+1 D_i,
// the same sweep products.  The mixed mode's inner FP32 steps (one A and one
// P apply each) are counted, and its outer preconditioner steps (each a whole
// inner solve) are not.
static void fill_counts(const wc4d_problem* P, wc4d_info* info) {
  const int64_t T = P->N + 1, N = P->N, k = P->o.k;
  const bool mixed = (P->o.precision == WC4D_PREC_MIXED);
  const int64_t nA = info->n_apply_A + (mixed ? info->inner_iters : 0);
  const int64_t nP = mixed ? info->inner_iters : info->n_apply_P;
  const bool pd = (P->o.precond == WC4D_PRECOND_PD);
  const bool exactS = pd && (P->o.shat == WC4D_SHAT_EXACT);
  const int64_t sweepM = (P->o.lhat == WC4D_LHAT_LM && !exactS) ? 2 * (N - N / k) : 0;
  info->n_R = nA * T;
  info->n_D = nA * T + (exactS ? 0 : nP * T);
  info->n_Dhat_inv = pd ? nP * T : 0;
  info->n_Rhat_inv = nP * T;
  info->n_M = nA * 2 * N + nP * sweepM;
  info->n_cov = info->n_R + info->n_D;
  info->n_trsm = info->n_Dhat_inv + info->n_Rhat_inv;
}

static int solve_minres(wc4d_problem* P, wc4d_info* info, bool use_x0) {
  const int64_t n = P->n;
  double* Vb[3] = {P->V, P->V + n, P->V + 2 * n};
  double* Zb[2] = {P->V + 3 * n, P->V + 4 * n};
  double* Wb[3] = {P->V + 5 * n, P->V + 6 * n, P->V + 7 * n};
  double* Az = P->V + 8 * n;
  const int* done = &P->stat->done;
  cudaStream_t st = P->st;
  // rhs norm
  dot_partial<double>(P->rhs, P->rhs, n, P->part3, nullptr, st);
  dot_finish(P->part3, P->scal, 1, st);
  WC4D_CUDA(cudaMemsetAsync(Vb[0], 0, sizeof(double) * n, st));
  WC4D_CUDA(cudaMemsetAsync(Wb[0], 0, sizeof(double) * n, st));
  WC4D_CUDA(cudaMemsetAsync(Wb[1], 0, sizeof(double) * n, st));
  int64_t nA = 0, nP = 0;
  if (use_x0) {
    apply_A<double>(P, P->f64, P->plan_A, P->x, Az, nullptr);
    vec_sub(P->rhs, Az, Vb[1], n, st);
    ++nA;
  } else {
    WC4D_CUDA(cudaMemsetAsync(P->x, 0, sizeof(double) * n, st));
    launch_copy_d(Vb[1], P->rhs, n, st);
  }
  apply_P<double>(P, WC4D_PRECOND_PD, P->f64, Vb[1], Zb[0], nullptr);
  ++nP;
  dot_partial<double>(Zb[0], Vb[1], n, P->part2, nullptr, st);
  minres_init(P->part2, P->sc, P->stat, P->o.tol, st);
  int it = 0;  // completed iterations
  int status = WC4D_OK;
  double relres = 1.0;
  bool converged = false;
  fetch_stat(P);
  if (P->h_stat->done) {
    status = P->h_stat->status;
    converged = (status == 0);
  }
  while (!converged && status == WC4D_OK) {
    const int batch = std::min(P->o.check_every, P->maxit - it);
    if (batch <= 0) break;
    for (int b = 0; b < batch; ++b) {
      const int j = it + b;
      double* v_old = Vb[j % 3];
      double* v = Vb[(j + 1) % 3];
      double* v_new = Vb[(j + 2) % 3];
      double* z = Zb[j % 2];
      double* z_new = Zb[(j + 1) % 2];
      double* w_old = Wb[j % 3];
      double* w = Wb[(j + 1) % 3];
      double* w_new = Wb[(j + 2) % 3];
      double* sc_in = P->sc + (j % 2) * MS_COUNT;
      double* sc_out = P->sc + ((j + 1) % 2) * MS_COUNT;
      apply_A<double>(P, P->f64, P->plan_A, z, Az, done);
      dot_partial<double>(Az, z, n, P->part, done, st);
      minres_v_update(P->part, sc_in, Az, v, v_old, v_new, n, done, st);
      apply_P<double>(P, WC4D_PRECOND_PD, P->f64, v_new, z_new, done);
      dot_partial<double>(z_new, v_new, n, P->part2, done, st);
      minres_update(P->part, P->part2, sc_in, sc_out, z, w_old, w, w_new, P->x, n, P->stat, st);
    }
    fetch_stat(P);
    it = P->h_stat->iters;
    if (P->h_stat->status != 0) {
      status = P->h_stat->status;
      break;
    }
    if (P->h_stat->done) {
      relres = true_relres(P, P->rhs, P->x);
      ++nA;
      if (!std::isfinite(relres)) {
        status = WC4D_ERR_NONFINITE;
        break;
      }
      if (relres <= P->o.tol || P->h_stat->est == 0.0) {
        converged = true;
        break;
      }
      // C12: the recurrence estimate met the tolerance but the true FP64
      // residual did not; tighten the estimate threshold and continue.
      resume_after_false_stop(P, P->h_stat->est, relres);
    } else if (it >= P->maxit) {
      break;
    }
  }
  nA += it;
  nP += it;
  if (!converged) {
    relres = true_relres(P, P->rhs, P->x);
    ++nA;
    if (status == WC4D_OK)
      status = !std::isfinite(relres) ? WC4D_ERR_NONFINITE : (relres <= P->o.tol ? WC4D_OK : WC4D_ERR_MAXIT);
  }
  if (info) {
    info->iters = it;
    info->relres_true = relres;
    info->relres_est = P->h_stat->est;
    info->n_apply_A = nA;
    info->n_apply_P = nP;
  }
  return status;
}

// MIXED preconditioner of the outer FGMRES: m steps of right-preconditioned
// GMRES on the FP32 copy of A with the FP32 copy of the chosen P, from a zero
// initial guess, on the outer Arnoldi vector v; z (FP64) = the inner iterate.
// Fixed step count (no inner convergence test), so every outer step applies
// the same amount of work; a lucky breakdown ends the inner loop early through
// the inner status flag.
static void inner_solve(wc4d_problem* P, const double* v, double* z) {
  const int64_t n = P->n;
  const int mi = P->mi, ldh = mi + 1;
  cudaStream_t st = P->st;
  const int* done = &P->stat_in->done;
  const int which = P->o.precond;
  vec_convert<float, double>(v, P->stage, n, 1.0, st);
  dot_partial<float>(P->stage, P->stage, n, P->part2i, nullptr, st);
  dot_finish(P->part2i, P->bnormi, 1, st);
  gm_init<float>(P->stage, P->part2i, P->Vi, P->gi, P->stat_in, 0.0, n, st);
  for (int j = 0; j < mi; ++j) {
    float* vj = P->Vi + (int64_t)j * n;
    float* zj = P->Zi + (int64_t)j * n;
    float* w = P->Vi + (int64_t)(j + 1) * n;
    apply_P<float>(P, which, P->f32, vj, zj, done);
    apply_A<float>(P, P->f32, P->plan_A, zj, w, done);
    gm_mdot<float>(P->Vi, n, j + 1, w, n, P->parti, done, st);
    gm_mdot_reduce(P->parti, j + 1, orth_chunks(n), P->h1i, done, st);
    gm_mupdate<float>(P->Vi, n, j + 1, P->h1i, w, n, done, st);
    gm_mdot<float>(P->Vi, n, j + 1, w, n, P->parti, done, st);
    gm_mdot_reduce(P->parti, j + 1, orth_chunks(n), P->h2i, done, st);
    gm_mupdate<float>(P->Vi, n, j + 1, P->h2i, w, n, done, st);
    dot_partial<float>(w, w, n, P->part2i, done, st);
    gm_hessenberg(j, P->h1i, P->h2i, P->part2i, P->Hi, ldh, P->csi, P->sni, P->gi, P->hnexti, P->stat_in, P->bnormi,
                  st);
    gm_normalize<float>(w, P->hnexti, w, n, done, st);
  }
  gm_solve_y_dev(P->Hi, ldh, P->gi, P->stat_in, mi, P->yi, st);
  gm_combine_dev<double, float>(P->Zi, n, P->stat_in, mi, P->yi, z, n, st);
  P->inner_total += mi;
}

// GMRES with the delayed-reorthogonalisation Arnoldi on the split basis (DF32
// mode).  Step j: Z~_j = P^-1 u_j, w = A Z~_j, one dot pass, the coefficient
// kernel (completes Hessenberg column j-1, Givens, status, column j of T), one
// update pass (q_j and u_{j+1}).  The solution is x0 + Z~ T^-1 y.
static int solve_gmres_dc(wc4d_problem* P, wc4d_info* info, bool use_x0) {
  const int64_t n = P->n;
  const int ldh = P->maxit + 1;
  cudaStream_t st = P->st;
  const int* done = &P->stat->done;
  const int which = P->o.precond;
  const int64_t lb = P->ldb;
  const bool p32 = (P->o.precision == WC4D_PREC_DF32_P32);
  int64_t nA = 0, nP = 0;
  dot_partial<double>(P->rhs, P->rhs, n, P->part3, nullptr, st);
  dot_finish(P->part3, P->scal, 1, st);
  WC4D_CUDA(cudaMemcpyAsync(P->bnorm, P->scal, sizeof(double), cudaMemcpyDeviceToDevice, st));
  double* r0 = P->V;
  if (use_x0) {
    launch_copy_d(P->x0, P->x, n, st);
    apply_A<double>(P, P->f64, P->plan_A, P->x0, r0, nullptr);
    vec_sub(P->rhs, r0, r0, n, st);
    ++nA;
  } else {
    launch_copy_d(r0, P->rhs, n, st);
  }
  dot_partial<double>(r0, r0, n, P->part2, nullptr, st);
  gm_init<double>(r0, P->part2, P->vcur, P->g, P->stat, P->o.tol, n, st);
  WC4D_CUDA(cudaMemcpyAsync(P->dcst + DC_BETA, P->g, sizeof(double), cudaMemcpyDeviceToDevice, st));
  gm_split_basis(P->vcur, P->Vh, P->Vl, n, P->b6, st);
  WC4D_CUDA(cudaMemsetAsync(P->H, 0, sizeof(double) * (size_t)ldh * P->maxit, st));
  WC4D_CUDA(cudaMemsetAsync(P->Hraw, 0, sizeof(double) * (size_t)ldh * P->maxit, st));
  int status = WC4D_OK;
  double relres = 1.0;
  bool converged = false;
  int it = 0;           // columns completed
  int next = 0;         // next Arnoldi step to run
  bool pending_update = false;
  fetch_stat(P);
  if (P->h_stat->done) {
    status = P->h_stat->status;
    if (status == 0) {
      converged = true;
      relres = 0.0;
      if (use_x0)
        launch_copy_d(P->x, P->x0, n, st);
      else
        WC4D_CUDA(cudaMemsetAsync(P->x, 0, sizeof(double) * n, st));
    }
  }
  while (!converged && status == WC4D_OK) {
    if (pending_update) {  // the step that stopped on a false convergence still owes its update pass
      gm_dc_update(P->Vh, P->Vl, lb, next - 1, P->ecoef, P->cprev, P->dcst, P->wbuf, P->vcur, n, P->Hraw, ldh,
                   P->hcbuf, nullptr, st, P->b6);
      pending_update = false;
    }
    const int batch = std::min(P->o.check_every, P->maxit + 1 - next);
    if (batch <= 0) break;
    for (int b = 0; b < batch; ++b) {
      const int j = next + b;
      double* zj = P->Z + (int64_t)j * n;
      if (p32) {  // FP32 preconditioner: the stored Z~_j is whatever it computed
        vec_convert<float, double>(P->vcur, P->stage, n, 1.0, st);
        apply_P<float>(P, which, P->f32, P->stage, P->zf, done);
        vec_convert<double, float>(P->zf, zj, n, 1.0, st);
      } else {
        apply_P<double>(P, which, P->f64, P->vcur, zj, done);
      }
      // w = A z_j, written with its double-float split for the dot pass
      apply_A<double>(P, P->f64, P->plan_A, zj, P->wbuf, done, P->wh, P->wl);
      float2* part2 = reinterpret_cast<float2*>(P->part);  // one double-float pair per (row, chunk)
      gm_dc_dot(P->Vh, P->Vl, lb, j, P->wh, P->wl, n, part2, done, st, P->b6);
      gm_dc_coef(j, part2, dc_dot_chunks(n, j + 1), P->dcst, P->bprev, P->cprev, P->ecoef, P->Hraw, P->H, P->Tm, ldh,
                 P->cs, P->sn, P->g, P->hnext, P->stat, P->bnorm, P->hcbuf, st);
      if (j < P->maxit)
        gm_dc_update(P->Vh, P->Vl, lb, j, P->ecoef, P->cprev, P->dcst, P->wbuf, P->vcur, n, P->Hraw, ldh,
                     P->hcbuf, done, st, P->b6);
    }
    fetch_stat(P);
    it = P->h_stat->iters;
    if (P->h_stat->status != 0) {
      status = P->h_stat->status;
      break;
    }
    const int ran_to = next + batch;  // steps next..ran_to-1 were issued
    if (P->h_stat->done || ran_to > P->maxit) {
      const int k = std::min(it, P->maxit);
      gm_solve_y(P->H, ldh, P->g, k, P->y, st);
      gm_solve_y(P->Tm, ldh, P->y, k, P->yhat, st);  // T yhat = y
      gm_combine<double, double>(P->Z, n, k, P->yhat, use_x0 ? P->x0 : nullptr, P->x, n, st);
      relres = true_relres(P, P->rhs, P->x);
      ++nA;
      if (!std::isfinite(relres)) {
        status = WC4D_ERR_NONFINITE;
        break;
      }
      if (relres <= P->o.tol) {
        converged = true;
        break;
      }
      if (!P->h_stat->done) break;  // maxit
      double hn = 0;
      WC4D_CUDA(cudaMemcpy(&hn, P->hnext, sizeof(double), cudaMemcpyDeviceToHost));
      if (hn == 0.0 || it >= P->maxit) {
        status = (it >= P->maxit) ? WC4D_OK : WC4D_ERR_BREAKDOWN;
        break;
      }
      resume_after_false_stop(P, P->h_stat->est, relres);
      next = it + 1;  // step `it` completed its coefficients; its update pass is pending
      pending_update = true;
    } else {
      next = ran_to;
    }
  }
  nA += it + 1;
  nP += it + 1;
  if (!converged && status == WC4D_OK) status = WC4D_ERR_MAXIT;
  if (info) {
    info->iters = it;
    info->relres_true = relres;
    info->relres_est = P->h_stat->est;
    info->n_apply_A = nA;
    info->n_apply_P = nP;
    info->inner_iters = 0;
  }
  return status;
}

static int solve_gmres(wc4d_problem* P, wc4d_info* info, bool use_x0) {
  if (P->dcgs) return solve_gmres_dc(P, info, use_x0);
  const int64_t n = P->n;
  const int ldh = P->maxit + 1;
  cudaStream_t st = P->st;
  const int* done = &P->stat->done;
  const int which = P->o.precond;
  double* x0 = use_x0 ? P->x0 : nullptr;  // kept for the final combination
  int64_t nA = 0, nP = 0;
  dot_partial<double>(P->rhs, P->rhs, n, P->part3, nullptr, st);
  dot_finish(P->part3, P->scal, 1, st);
  WC4D_CUDA(cudaMemcpyAsync(P->bnorm, P->scal, sizeof(double), cudaMemcpyDeviceToDevice, st));
  const bool sb = P->split_basis;
  double* r0 = sb ? P->V : P->V + n;  // V[1] is free until the first Arnoldi step
  if (use_x0) {
    launch_copy_d(x0, P->x, n, st);
    apply_A<double>(P, P->f64, P->plan_A, x0, r0, nullptr);
    vec_sub(P->rhs, r0, r0, n, st);
    ++nA;
  } else {
    launch_copy_d(r0, P->rhs, n, st);
  }
  dot_partial<double>(r0, r0, n, P->part2, nullptr, st);
  gm_init<double>(r0, P->part2, sb ? P->vcur : P->V, P->g, P->stat, P->o.tol, n, st);
  if (sb) gm_split(P->vcur, P->Vh, P->Vl, n, nullptr, st);
  WC4D_CUDA(cudaMemsetAsync(P->H, 0, sizeof(double) * (size_t)ldh * P->maxit, st));
  int it = 0;
  int status = WC4D_OK;
  double relres = 1.0;
  bool converged = false;
  fetch_stat(P);
  if (P->h_stat->done) {
    status = P->h_stat->status;
    if (status == 0) {
      converged = true;
      relres = 0.0;
      launch_copy_d(P->x, use_x0 ? x0 : P->x, n, st);
      if (!use_x0) WC4D_CUDA(cudaMemsetAsync(P->x, 0, sizeof(double) * n, st));
    }
  }
  bool need_normalize = false;
  while (!converged && status == WC4D_OK) {
    const int batch = std::min(P->o.check_every, P->maxit - it);
    if (batch <= 0) break;
    if (need_normalize) {
      if (sb)
        gm_normalize_df(P->wbuf, P->hnext, P->vcur, P->Vh + (int64_t)it * P->ldb, P->Vl + (int64_t)it * P->ldb, n,
                        nullptr, st);
      else
        gm_normalize<double>(P->V + (int64_t)it * n, P->hnext, P->V + (int64_t)it * n, n, nullptr, st);
      need_normalize = false;
    }
    for (int b = 0; b < batch; ++b) {
      const int j = it + b;
      double* vj = sb ? P->vcur : P->V + (int64_t)j * n;
      double* zj = P->Z + (int64_t)j * n;
      double* w = sb ? P->wbuf : P->V + (int64_t)(j + 1) * n;
      if (sb) {
        if (P->o.precision == WC4D_PREC_MIXED)
          inner_solve(P, vj, zj);
        else
          apply_P<double>(P, which, P->f64, vj, zj, done);
        apply_A<double>(P, P->f64, P->plan_A, zj, w, done);
        const int nc = dot_chunks(n, j + 1);
        gm_split(w, P->wh, P->wl, n, done, st);
        const int64_t lb = P->ldb;
        gm_mdot_df(P->Vh, P->Vl, lb, j + 1, P->wh, P->wl, n, P->part, done, st);
        gm_mdot_reduce(P->part, j + 1, nc, P->h1, done, st);
        gm_mupdate_df(P->Vh, P->Vl, lb, j + 1, P->h1, w, P->wh, P->wl, n, done, st);
        gm_mdot_df(P->Vh, P->Vl, lb, j + 1, P->wh, P->wl, n, P->part, done, st);
        gm_mdot_reduce(P->part, j + 1, nc, P->h2, done, st);
        gm_mupdate_df(P->Vh, P->Vl, lb, j + 1, P->h2, w, P->wh, P->wl, n, done, st);
        dot_partial<double>(w, w, n, P->part2, done, st);
        gm_hessenberg(j, P->h1, P->h2, P->part2, P->H, ldh, P->cs, P->sn, P->g, P->hnext, P->stat, P->bnorm, st);
        gm_normalize_df(w, P->hnext, P->vcur, P->Vh + (int64_t)(j + 1) * P->ldb, P->Vl + (int64_t)(j + 1) * P->ldb, n,
                        done, st);
        continue;
      }
      if (P->o.precision == WC4D_PREC_MIXED)
        inner_solve(P, vj, zj);
      else
        apply_P<double>(P, which, P->f64, vj, zj, done);
      apply_A<double>(P, P->f64, P->plan_A, zj, w, done);
      gm_mdot<double>(P->V, n, j + 1, w, n, P->part, done, st);
      gm_mdot_reduce(P->part, j + 1, orth_chunks(n), P->h1, done, st);
      gm_mupdate<double>(P->V, n, j + 1, P->h1, w, n, done, st);
      gm_mdot<double>(P->V, n, j + 1, w, n, P->part, done, st);
      gm_mdot_reduce(P->part, j + 1, orth_chunks(n), P->h2, done, st);
      gm_mupdate<double>(P->V, n, j + 1, P->h2, w, n, done, st);
      dot_partial<double>(w, w, n, P->part2, done, st);
      gm_hessenberg(j, P->h1, P->h2, P->part2, P->H, ldh, P->cs, P->sn, P->g, P->hnext, P->stat, P->bnorm, st);
      gm_normalize<double>(w, P->hnext, w, n, done, st);
    }
    fetch_stat(P);
    it = P->h_stat->iters;
    if (P->h_stat->status != 0) {
      status = P->h_stat->status;
      break;
    }
    if (P->h_stat->done || it >= P->maxit) {
      gm_solve_y(P->H, ldh, P->g, it, P->y, st);
      gm_combine<double, double>(P->Z, n, it, P->y, x0, P->x, n, st);
      relres = true_relres(P, P->rhs, P->x);
      ++nA;
      if (!std::isfinite(relres)) {
        status = WC4D_ERR_NONFINITE;
        break;
      }
      if (relres <= P->o.tol) {
        converged = true;
        break;
      }
      if (it >= P->maxit) break;
      double hn = 0;
      WC4D_CUDA(cudaMemcpy(&hn, P->hnext, sizeof(double), cudaMemcpyDeviceToHost));
      if (hn == 0.0) {
        status = WC4D_ERR_BREAKDOWN;
        break;
      }
      resume_after_false_stop(P, P->h_stat->est, relres);
      need_normalize = true;
    }
  }
  nA += it;
  nP += it;
  if (!converged && status == WC4D_OK) status = WC4D_ERR_MAXIT;
  if (info) {
    info->iters = it;
    info->relres_true = relres;
    info->relres_est = P->h_stat->est;
    info->n_apply_A = nA;
    info->n_apply_P = nP;
    info->inner_iters = (int)P->inner_total;
  }
  return status;
}

void l96_forecast(const double* in, double* out, int count, int s, double F, double dt, int steps, cudaStream_t st);
void l96_background(const double* xb, double* traj, int N, int s, double F, double dt, int steps, cudaStream_t st);
void l96_tlm_bands(const double* traj, double* bands, int N, int s, int lo, int hi, double F, double dt, int steps,
                   cudaStream_t st);
void gn_rhs(const double* xb, const double* traj, const double* fc, const double* y, const int* obs, int s, int N,
            int p, double* rhs, cudaStream_t st);

static void l96_check(wc4d_problem* P, const wc4d_l96_params* prm) {
  WC4D_CHECK(prm != nullptr, WC4D_ERR_ARG, "null parameters");
  WC4D_CHECK(P->md.kind == WC4D_MODEL_BANDED, WC4D_ERR_ARG, "Gauss-Newton for Lorenz-96 needs a BANDED problem");
  WC4D_CHECK(!P->pertime, WC4D_ERR_ARG, "the Lorenz-96 calls observe one set at every time (no per-time sets)");
  WC4D_CHECK(prm->steps_per_obs >= 1 && prm->outer_loops >= 0 && prm->dt > 0, WC4D_ERR_ARG, "bad L96 parameters");
  WC4D_CHECK(P->md.lo == 8 * prm->steps_per_obs && P->md.hi == 4 * prm->steps_per_obs, WC4D_ERR_ARG,
             "band offsets must be lo = 8 steps, hi = 4 steps");
  WC4D_CHECK(P->s <= 4096, WC4D_ERR_ARG, "Lorenz-96 kernels keep the state in shared memory: s <= 4096");
  WC4D_CHECK(P->md.lo + P->md.hi + 1 <= P->s, WC4D_ERR_ARG, "band wider than the state: colours would alias");
}

static void l96_linearize(wc4d_problem* P, const wc4d_l96_params* prm, const double* xb_in, const double* y_in,
                          const double* traj_in, int mem_kind, double* rhs_out) {
  l96_check(P, prm);
  const int s = P->s, N = P->N, p = P->p;
  cudaStream_t st = P->st;
  double *xb = nullptr, *y = nullptr, *traj = nullptr, *fc = nullptr;
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    cudaFree(xb);
    cudaFree(y);
    cudaFree(traj);
    cudaFree(fc);
  };
  try {
    WC4D_CUDA(cudaMalloc(&xb, sizeof(double) * s));
    WC4D_CUDA(cudaMalloc(&y, sizeof(double) * P->np));
    WC4D_CUDA(cudaMalloc(&traj, sizeof(double) * P->ns));
    WC4D_CUDA(cudaMalloc(&fc, sizeof(double) * std::max<int64_t>(1, (int64_t)N * s)));
    copy_in(xb, xb_in, sizeof(double) * s, mem_kind, st);
    copy_in(y, y_in, sizeof(double) * P->np, mem_kind, st);
    copy_in(traj, traj_in, sizeof(double) * P->ns, mem_kind, st);
    l96_tlm_bands(traj, P->d_bands, N, s, P->md.lo, P->md.hi, prm->forcing, prm->dt, prm->steps_per_obs, st);
    if (N > 0) l96_forecast(traj, fc, N, s, prm->forcing, prm->dt, prm->steps_per_obs, st);
    gn_rhs(xb, traj, fc, y, P->d_obs, s, N, p, P->rhs, st);
    WC4D_CUDA(cudaMemcpyAsync(rhs_out, P->rhs, sizeof(double) * P->n,
                              mem_kind == WC4D_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    WC4D_CUDA(cudaStreamSynchronize(st));
  } catch (...) {
    cleanup();
    throw;
  }
  cleanup();
}

static int l96_gauss_newton(wc4d_problem* P, const wc4d_l96_params* prm, const double* xb_in, const double* y_in,
                            double* traj_io, bool init_bg, int mem_kind, wc4d_info* infos) {
  l96_check(P, prm);
  const int s = P->s, N = P->N, p = P->p;
  cudaStream_t st = P->st;
  std::vector<void*> tmp;
  auto dalloc = [&](int64_t cnt) {
    void* q = nullptr;
    if (cudaMalloc(&q, sizeof(double) * (size_t)std::max<int64_t>(cnt, 1)) != cudaSuccess)
      throw Error{WC4D_ERR_NOMEM, "cudaMalloc failed in Gauss-Newton"};
    tmp.push_back(q);
    return (double*)q;
  };
  int status = WC4D_OK;
  try {
    double* xb = dalloc(s);
    double* y = dalloc(P->np);
    double* traj = dalloc(P->ns);
    double* fc = dalloc((int64_t)N * s);
    copy_in(xb, xb_in, sizeof(double) * s, mem_kind, st);
    copy_in(y, y_in, sizeof(double) * P->np, mem_kind, st);
    if (init_bg)
      l96_background(xb, traj, N, s, prm->forcing, prm->dt, prm->steps_per_obs, st);
    else
      copy_in(traj, traj_io, sizeof(double) * P->ns, mem_kind, st);
    for (int l = 0; l < prm->outer_loops; ++l) {
      l96_tlm_bands(traj, P->d_bands, N, s, P->md.lo, P->md.hi, prm->forcing, prm->dt, prm->steps_per_obs, st);
      if (N > 0) l96_forecast(traj, fc, N, s, prm->forcing, prm->dt, prm->steps_per_obs, st);
      gn_rhs(xb, traj, fc, y, P->d_obs, s, N, p, P->rhs, st);
      wc4d_info loc{};
      P->inner_total = 0;
      const auto t0 = std::chrono::steady_clock::now();
      const int rc = (P->o.krylov == WC4D_KRYLOV_MINRES) ? solve_minres(P, &loc, false) : solve_gmres(P, &loc, false);
      loc.status = rc;
      loc.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      if (infos) infos[l] = loc;
      // x^(l+1) = x^(l) + dx  (dx = third block of the solution)
      vec_axpby<double>(traj, P->x + P->ns + P->np, 1.0, 1.0, P->ns, st);
      if (rc != WC4D_OK) {
        status = rc;
        break;
      }
    }
    WC4D_CUDA(cudaMemcpyAsync(traj_io, traj, sizeof(double) * P->ns,
                              mem_kind == WC4D_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    WC4D_CUDA(cudaStreamSynchronize(st));
  } catch (...) {
    cudaStreamSynchronize(st);
    for (void* q : tmp) cudaFree(q);
    throw;
  }
  for (void* q : tmp) cudaFree(q);
  return status;
}

// d_t[r] = traj_t[obs[r]] + E[r + t p]
__global__ void obs_rhs_kernel(const double* traj, const double* E, const int* obs, int s, int p, int N, double* d) {
  const int64_t total = (int64_t)(N + 1) * p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(e / p), r = (int)(e % p);
    d[e] = traj[(int64_t)t * s + obs[r]] + E[e];
  }
}

static void synthesize_rhs(wc4d_problem* P, const double* zb_in, const double* zr_in, int mem_kind, double* rhs_out) {
  WC4D_CHECK(P->md.kind == WC4D_MODEL_STENCIL3, WC4D_ERR_ARG, "synthesize_rhs needs a linear (STENCIL3) model");
  WC4D_CHECK(!P->pertime, WC4D_ERR_ARG, "synthesize_rhs observes one set at every time (no per-time sets)");
  WC4D_CHECK(!P->band, WC4D_ERR_ARG, "synthesize_rhs needs dense B (not the banded modified SOAR)");
  const int s = P->s, p = P->p, N = P->N;
  cudaStream_t st = P->st;
  const int mmax = std::max(s, p);
  std::vector<void*> tmp;
  auto dalloc = [&](int64_t cnt) {
    void* q = nullptr;
    if (cudaMalloc(&q, sizeof(double) * (size_t)std::max<int64_t>(cnt, 1)) != cudaSuccess)
      throw Error{WC4D_ERR_NOMEM, "cudaMalloc failed in synthesize_rhs"};
    tmp.push_back(q);
    return (double*)q;
  };
  try {
    double* zb = dalloc(s);
    double* zr = dalloc(P->np);
    copy_in(zb, zb_in, sizeof(double) * s, mem_kind, st);
    copy_in(zr, zr_in, sizeof(double) * P->np, mem_kind, st);
    double* work = dalloc((int64_t)mmax * mmax);
    double* Lt = dalloc((int64_t)mmax * mmax);
    double* scratch = dalloc((int64_t)mmax * 64 + 64 * 64 * 2);
    int* info = (int*)dalloc(1);
    double* rhs = dalloc(P->n);
    WC4D_CUDA(cudaMemsetAsync(rhs, 0, sizeof(double) * P->n, st));
    // u = chol(B) z_b, then the background-minus-truth trajectory M^t (-u)
    launch_copy_d(work, P->f64.B, (int64_t)s * s, st);
    WC4D_CUDA(cudaMemsetAsync(info, 0, sizeof(int), st));
    cholesky(work, s, info, st, scratch);
    WC4D_CHECK(read_flag(info, st) == 0, WC4D_ERR_NOT_SPD, "Cholesky of B failed");
    launch_transpose(work, Lt, s, st);
    double* traj = dalloc(P->ns);
    WC4D_CUDA(cudaMemsetAsync(traj, 0, sizeof(double) * P->ns, st));
    gemm_once(P, Lt, s, zb, s, s, s, 1, traj, s, EPI_NEG_STORE);
    lhat_sweep<double>(P->md, N + 1, traj, traj, false, false, nullptr, st);
    // E = chol(R) Z_r
    launch_copy_d(work, P->f64.R, (int64_t)p * p, st);
    WC4D_CUDA(cudaMemsetAsync(info, 0, sizeof(int), st));
    cholesky(work, p, info, st, scratch);
    WC4D_CHECK(read_flag(info, st) == 0, WC4D_ERR_NOT_SPD, "Cholesky of R failed");
    launch_transpose(work, Lt, p, st);
    double* E = dalloc(P->np);
    gemm_once(P, Lt, p, zr, p, p, p, N + 1, E, p, EPI_STORE);
    const int nb = (int)std::min<int64_t>((P->np + 255) / 256, 152 * 8);
    obs_rhs_kernel<<<nb, 256, 0, st>>>(traj, E, P->d_obs, s, p, N, rhs + P->ns);
    WC4D_LAUNCH_CHECK();
    WC4D_CUDA(cudaMemcpyAsync(rhs_out, rhs, sizeof(double) * P->n,
                              mem_kind == WC4D_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    WC4D_CUDA(cudaStreamSynchronize(st));
  } catch (...) {
    cudaStreamSynchronize(st);
    for (void* q : tmp) cudaFree(q);
    throw;
  }
  for (void* q : tmp) cudaFree(q);
}

}  // namespace wc4d

// ================================================================ C ABI
#define WC4D_API_BEGIN try {
#define WC4D_API_END                                   \
  }                                                    \
  catch (const wc4d::Error& e) {                       \
    wc4d::set_error(e.msg);                            \
    return e.code;                                     \
  }                                                    \
  catch (const std::exception& e) {                    \
    wc4d::set_error(std::string("exception: ") + e.what()); \
    return WC4D_ERR_CUDA;                              \
  }                                                    \
  catch (...) {                                        \
    wc4d::set_error("unknown exception");              \
    return WC4D_ERR_CUDA;                              \
  }

extern "C" {

void wc4d_default_opts(wc4d_solve_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precond = WC4D_PRECOND_PI;
  o->k = 1;
  o->rhat = WC4D_RHAT_EXACT;
  o->kappa_max = 100.0;
  o->shat = WC4D_SHAT_PAPER;
  o->dhat = WC4D_DHAT_EXACT;
  o->dhat_delta = 0.01;
  o->krylov = WC4D_KRYLOV_GMRES;
  o->tol = 1e-6;
  o->maxit = 1000;
  o->precision = WC4D_PREC_FP64;
  o->inner_iters = 20;
  o->check_every = 4;
}

int wc4d_setup_problem(const wc4d_problem_desc* desc, const wc4d_solve_opts* opts, void* cuda_stream,
                       wc4d_problem** out) {
  WC4D_API_BEGIN
  WC4D_CHECK(out != nullptr, WC4D_ERR_ARG, "out is null");
  *out = nullptr;
  wc4d_problem* P = new wc4d_problem();
  P->st = (cudaStream_t)cuda_stream;
  try {
    setup(P, desc, opts);
  } catch (...) {
    cudaStreamSynchronize(P->st);
    delete P;
    throw;
  }
  *out = P;
  return WC4D_OK;
  WC4D_API_END
}

int wc4d_apply_saddle(wc4d_problem* P, const double* v, double* out) {
  WC4D_API_BEGIN
  WC4D_CHECK(P && v && out, WC4D_ERR_ARG, "null argument");
  apply_A<double>(P, P->f64, P->plan_A, v, out, nullptr);
  return WC4D_OK;
  WC4D_API_END
}

int wc4d_status(wc4d_problem* P) {
  WC4D_API_BEGIN
  WC4D_CHECK(P, WC4D_ERR_ARG, "null argument");
  WC4D_CUDA(cudaStreamSynchronize(P->st));
  check_kernel_waits(P);
  return WC4D_OK;
  WC4D_API_END
}

void wc4d_set_wait_limit_ns(uint64_t ns) { oz_set_wait_limit((unsigned long long)ns); }

int wc4d_apply_precond(wc4d_problem* P, int32_t which, const double* v, double* out) {
  WC4D_API_BEGIN
  WC4D_CHECK(P && v && out, WC4D_ERR_ARG, "null argument");
  WC4D_CHECK(which == WC4D_PRECOND_PD || which == WC4D_PRECOND_PI, WC4D_ERR_ARG, "bad preconditioner");
  WC4D_CHECK(which == WC4D_PRECOND_PI || P->have_pd, WC4D_ERR_ARG,
             "P_D needs a problem set up with precond = PD (Dhat factors)");
  apply_P<double>(P, which, P->f64, v, out, nullptr);
  return WC4D_OK;
  WC4D_API_END
}

int wc4d_solve(wc4d_problem* P, const double* rhs, double* x, int32_t use_x0, int32_t mem_kind, wc4d_info* info) {
  WC4D_API_BEGIN
  wc4d::NvtxRange nvtx_range("wc4d.solve");
  WC4D_CHECK(P && rhs && x, WC4D_ERR_ARG, "null argument");
  WC4D_CHECK(mem_kind == WC4D_MEM_HOST || mem_kind == WC4D_MEM_DEVICE, WC4D_ERR_ARG, "bad mem_kind");
  const auto t0 = std::chrono::steady_clock::now();
  const size_t bytes = sizeof(double) * (size_t)P->n;
  const cudaMemcpyKind kin = mem_kind == WC4D_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind kout = mem_kind == WC4D_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  WC4D_CUDA(cudaMemcpyAsync(P->rhs, rhs, bytes, kin, P->st));
  if (use_x0) WC4D_CUDA(cudaMemcpyAsync(P->x, x, bytes, kin, P->st));
  wc4d_info loc{};
  P->inner_total = 0;
  int status;
  if (P->o.krylov == WC4D_KRYLOV_MINRES)
    status = solve_minres(P, &loc, use_x0 != 0);
  else
    status = solve_gmres(P, &loc, use_x0 != 0);
  if (status != WC4D_OK && P->net_on) {
    // the plain Schur block is the fallback of the learned one
    P->net_on = false;
    if (use_x0) WC4D_CUDA(cudaMemcpyAsync(P->x, x, bytes, kin, P->st));
    loc = wc4d_info{};
    try {
      status = solve_gmres(P, &loc, use_x0 != 0);
    } catch (...) {
      P->net_on = true;
      throw;
    }
    P->net_on = true;
    loc.precond_fallback = 1;
  }
  WC4D_CUDA(cudaMemcpyAsync(x, P->x, bytes, kout, P->st));
  WC4D_CUDA(cudaStreamSynchronize(P->st));
  check_kernel_waits(P);
  fill_counts(P, &loc);
  loc.status = status;
  loc.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = loc;
  if (status != WC4D_OK) {
    char buf[200];
    snprintf(buf, sizeof buf, "solve ended with status %d after %d iterations (true relres %.3e)", status, loc.iters,
             loc.relres_true);
    wc4d::set_error(buf);
  }
  return status;
  WC4D_API_END
}

// ------------------------------------------------------------ learned block
static const char kNetMagic[8] = {'W', 'C', '4', 'D', 'N', 'E', 'T', '1'};

void wc4d_default_train_opts(wc4d_train_opts* o) {
  if (!o) return;
  o->pairs = 50000;
  o->hidden = 32;
  o->batch = 64;
  o->epochs = 4;
  o->lr = 1e-3;
  o->val_frac = 0.05;
  o->seed = 1;
  o->loss = WC4D_LOSS_ERROR;
}

int64_t wc4d_net_nparams(int32_t C, int32_t hidden) { return NetShape{C, hidden, 1}.nparams(); }

// Initial weights: uniform in +-1/sqrt(fan_in) from SplitMix64 of the seed
// (host), biases zero, the last layer scaled by 0.1 (a small first correction).
static std::vector<float> net_init(const NetShape& sh, uint64_t seed) {
  std::vector<float> w((size_t)sh.nparams(), 0.f);
  uint64_t z = seed * 0x9E3779B97F4A7C15ull + 12345;
  auto next = [&]() {
    z += 0x9E3779B97F4A7C15ull;
    uint64_t x = z;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    return (double)(x >> 11) * (1.0 / 9007199254740992.0);
  };
  for (int l = 0; l < NET_LAYERS; ++l) {
    const double a = 1.0 / std::sqrt((double)sh.ci(l) * NET_KW) * (l == NET_LAYERS - 1 ? 0.1 : 1.0);
    const int64_t nw = (int64_t)sh.co(l) * sh.ci(l) * NET_KW;
    for (int64_t i = 0; i < nw; ++i) w[(size_t)(sh.w_off(l) + i)] = (float)((2.0 * next() - 1.0) * a);
  }
  return w;
}

// Mean of |yn + f - tn|^2 / |tn|^2 over samples [i0, i1) of the pair store
// (with_net = 0: f = 0, the plain block), forward passes in batches of B.
static double net_val_error(wc4d_problem* P, const NetShape& sh, const float* params, const float* yn, const float* tn,
                            const double* tn2, int i0, int i1, int B, float* xb, float* acts[3], float* outb,
                            float* gout, int* d_idx, double* d_loss, bool with_net) {
  cudaStream_t st = P->st;
  const int64_t len = (int64_t)sh.C * sh.s;
  WC4D_CUDA(cudaMemsetAsync(d_loss, 0, sizeof(double), st));
  std::vector<int> idx(B);
  for (int b0 = i0; b0 < i1; b0 += B) {
    const int nb = std::min(B, i1 - b0);
    for (int b = 0; b < nb; ++b) idx[b] = b0 + b;
    WC4D_CUDA(cudaMemcpy(d_idx, idx.data(), sizeof(int) * nb, cudaMemcpyHostToDevice));
    net_gather(yn, d_idx, nb, len, xb, st);
    net_gather(tn, d_idx, nb, len, gout, st);  // targets into the gradient buffer (scratch here)
    if (with_net)
      net_forward(sh, params, nb, xb, acts, outb, st);
    else
      WC4D_CUDA(cudaMemsetAsync(outb, 0, sizeof(float) * nb * len, st));
    // loss kernel overwrites its gradient argument: give it acts[0] as scratch (>= nb * len floats)
    net_loss_grad(sh, nb, xb, outb, gout, tn2, d_idx, acts[0], d_loss, st);
  }
  double h = 0;
  WC4D_CUDA(cudaMemcpy(&h, d_loss, sizeof(double), cudaMemcpyDeviceToHost));
  return h / std::max(1, i1 - i0);
}

static void save_net(const char* path, const NetShape& sh, const std::vector<float>& w, double ve, double vp) {
  std::ofstream f(path, std::ios::binary);
  WC4D_CHECK(f.good(), WC4D_ERR_IO, std::string("cannot write ") + path);
  const int32_t hdr[3] = {sh.C, sh.H, sh.s};
  const int64_t np = sh.nparams();
  f.write(kNetMagic, 8);
  f.write((const char*)hdr, sizeof hdr);
  f.write((const char*)&np, sizeof np);
  f.write((const char*)w.data(), sizeof(float) * w.size());
  f.write((const char*)&ve, sizeof ve);
  f.write((const char*)&vp, sizeof vp);
  WC4D_CHECK(f.good(), WC4D_ERR_IO, std::string("write failed: ") + path);
}

int wc4d_precond_set_net(wc4d_problem* P, int32_t hidden, const float* params, int32_t active) {
  WC4D_API_BEGIN
  WC4D_CHECK(P && params, WC4D_ERR_ARG, "null argument");
  WC4D_CHECK(P->o.shat == WC4D_SHAT_LEARNED && P->net_params, WC4D_ERR_ARG,
             "the problem was not set up with shat = LEARNED");
  WC4D_CHECK(hidden >= 1 && hidden <= 64, WC4D_ERR_ARG, "hidden must lie in [1, 64]");
  P->net_sh = NetShape{P->N + 1, hidden, P->s};
  WC4D_CUDA(cudaMemcpyAsync(P->net_params, params, sizeof(float) * P->net_sh.nparams(), cudaMemcpyHostToDevice, P->st));
  WC4D_CUDA(cudaStreamSynchronize(P->st));
  P->net_on = active != 0;
  return WC4D_OK;
  WC4D_API_END
}

int wc4d_precond_load(wc4d_problem* P, const char* path) {
  WC4D_API_BEGIN
  WC4D_CHECK(P && path, WC4D_ERR_ARG, "null argument");
  WC4D_CHECK(P->o.shat == WC4D_SHAT_LEARNED && P->net_params, WC4D_ERR_ARG,
             "the problem was not set up with shat = LEARNED");
  std::ifstream f(path, std::ios::binary);
  WC4D_CHECK(f.good(), WC4D_ERR_IO, std::string("cannot read ") + path);
  char mg[8];
  int32_t hdr[3];
  int64_t np = 0;
  f.read(mg, 8);
  f.read((char*)hdr, sizeof hdr);
  f.read((char*)&np, sizeof np);
  WC4D_CHECK(f.good() && std::memcmp(mg, kNetMagic, 8) == 0, WC4D_ERR_IO, "not a wc4d network checkpoint");
  WC4D_CHECK(hdr[0] == P->N + 1 && hdr[2] == P->s && hdr[1] >= 1 && hdr[1] <= 64, WC4D_ERR_ARG,
             "checkpoint was trained for another (N+1, s)");
  const NetShape sh{hdr[0], hdr[1], hdr[2]};
  WC4D_CHECK(np == sh.nparams(), WC4D_ERR_IO, "checkpoint parameter count mismatch");
  std::vector<float> w((size_t)np);
  double ve = 0, vp = 0;
  f.read((char*)w.data(), sizeof(float) * np);
  f.read((char*)&ve, sizeof ve);
  f.read((char*)&vp, sizeof vp);
  WC4D_CHECK(f.good(), WC4D_ERR_IO, "truncated checkpoint");
  return wc4d_precond_set_net(P, sh.H, w.data(), ve < vp ? 1 : 0);
  WC4D_API_END
}

int wc4d_precond_train(wc4d_problem* P, const wc4d_train_opts* o_in, const char* ckpt_path, wc4d_train_report* rep) {
  WC4D_API_BEGIN
  WC4D_CHECK(P, WC4D_ERR_ARG, "null problem");
  wc4d_train_opts o;
  if (o_in)
    o = *o_in;
  else
    wc4d_default_train_opts(&o);
  WC4D_CHECK(P->o.shat == WC4D_SHAT_LEARNED && P->have_pd && P->o.rhat == WC4D_RHAT_EXACT &&
                 P->o.dhat == WC4D_DHAT_EXACT,
             WC4D_ERR_ARG, "training needs a problem set up with precond = PD, shat = LEARNED, rhat = dhat = EXACT");
  WC4D_CHECK(o.pairs >= 2 && o.hidden >= 1 && o.hidden <= 64 && o.batch >= 1 && o.batch <= 4096 && o.epochs >= 1 &&
                 o.lr > 0 && o.val_frac > 0 && o.val_frac < 1 &&
                 (o.loss == WC4D_LOSS_ERROR || o.loss == WC4D_LOSS_RESIDUAL),
             WC4D_ERR_ARG, "bad training options");
  cudaStream_t st = P->st;
  const int C = P->N + 1, s = P->s;
  const NetShape sh{C, o.hidden, s};
  const int64_t len = (int64_t)C * s, n = P->n;
  const int nval = std::max(1, (int)std::lround(o.pairs * o.val_frac));
  const int ntr = o.pairs - nval;
  WC4D_CHECK(ntr >= 1, WC4D_ERR_ARG, "no training pairs left after the validation split");
  std::vector<void*> owned;
  auto dalloc = [&](size_t bytes) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) throw wc4d::Error{WC4D_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e)};
    owned.push_back(p);
    return p;
  };
  const bool was_on = P->net_on;
  try {
    P->net_on = false;  // pairs use the plain operators
    float* yn = (float*)dalloc(sizeof(float) * len * o.pairs);
    float* tn = (float*)dalloc(sizeof(float) * len * o.pairs);
    double* tn2 = (double*)dalloc(sizeof(double) * o.pairs);
    double* va = (double*)dalloc(sizeof(double) * n);
    double* vb = (double*)dalloc(sizeof(double) * n);
    double* vc = (double*)dalloc(sizeof(double) * n);
    double* nrm2 = (double*)dalloc(sizeof(double));
    double* part = (double*)dalloc(sizeof(double) * DOT_BLOCKS);
    double* r2 = (double*)dalloc(sizeof(double) * o.pairs);   // |r|^2 per pair
    double* nu2 = (double*)dalloc(sizeof(double) * o.pairs);  // |y|^2 per pair
    WC4D_CUDA(cudaMemsetAsync(tn2, 0, sizeof(double) * o.pairs, st));
    const int64_t off3 = P->ns + P->np;  // the x block (Schur block) of a saddle vector
    const auto t0 = std::chrono::steady_clock::now();
    for (int i = 0; i < o.pairs; ++i) {
      // v: white noise, or S_hat^{-1} of white noise (alternately)
      WC4D_CUDA(cudaMemsetAsync(va, 0, sizeof(double) * n, st));
      normal_fill(va + off3, len, o.seed, (uint64_t)i * (uint64_t)len, st);
      if (i & 1) {
        apply_P<double>(P, WC4D_PRECOND_PD, P->f64, va, vb, nullptr);  // (0, 0, S_hat^{-1} xi)
      } else {
        launch_copy_d(vb, va, n, st);
      }
      // r = S v: A (0,0,v) = (L v, H v, 0); P_D of that = (D^-1 L v, R^-1 H v, 0); A of that: x block = S v
      apply_A<double>(P, P->f64, P->plan_A, vb, vc, nullptr);
      WC4D_CUDA(cudaMemsetAsync(vc + off3, 0, sizeof(double) * len, st));
      apply_P<double>(P, WC4D_PRECOND_PD, P->f64, vc, va, nullptr);
      WC4D_CUDA(cudaMemsetAsync(va + off3, 0, sizeof(double) * len, st));
      apply_A<double>(P, P->f64, P->plan_A, va, vc, nullptr);
      // y = S_hat^{-1} r
      dot_partial<double>(vc + off3, vc + off3, len, part, nullptr, st);
      dot_finish(part, r2 + i, 0, st);
      WC4D_CUDA(cudaMemsetAsync(va, 0, sizeof(double) * off3, st));
      launch_copy_d(va + off3, vc + off3, len, st);
      apply_P<double>(P, WC4D_PRECOND_PD, P->f64, va, vc, nullptr);
      dot_partial<double>(vc + off3, vc + off3, len, part, nullptr, st);
      dot_finish(part, nrm2, 0, st);
      WC4D_CUDA(cudaMemcpyAsync(nu2 + i, nrm2, sizeof(double), cudaMemcpyDeviceToDevice, st));
      net_store_pair(vc + off3, vb + off3, nrm2, yn + (int64_t)i * len, tn + (int64_t)i * len, tn2 + i, len, st);
    }
    WC4D_CUDA(cudaStreamSynchronize(st));
    const auto t1 = std::chrono::steady_clock::now();
    // |S tn|^2 = |r|^2 / |y|^2 per pair (the residual loss's normaliser)
    std::vector<double> hr2(o.pairs), hnu2(o.pairs), rn2(o.pairs);
    WC4D_CUDA(cudaMemcpy(hr2.data(), r2, sizeof(double) * o.pairs, cudaMemcpyDeviceToHost));
    WC4D_CUDA(cudaMemcpy(hnu2.data(), nu2, sizeof(double) * o.pairs, cudaMemcpyDeviceToHost));
    for (int i = 0; i < o.pairs; ++i) rn2[i] = hr2[i] / std::max(hnu2[i], 1e-300);
    const bool resid_loss = (o.loss == WC4D_LOSS_RESIDUAL);
    double* sd = (double*)dalloc(sizeof(double) * len);   // S d
    double* ssd = (double*)dalloc(sizeof(double) * len);  // S S d
    double* dd = (double*)dalloc(sizeof(double) * len);   // d
    double* lossv = (double*)dalloc(sizeof(double) * std::max(2, o.batch));
    // S x for an x block (time levels x grid): A (0,0,x) = (L x, H x, 0), P_D of
    // that = (D^-1 L x, R^-1 H x, 0), A again: its x block is S x
    auto applyS = [&](const double* x, double* out) {
      WC4D_CUDA(cudaMemsetAsync(va, 0, sizeof(double) * off3, st));
      launch_copy_d(va + off3, x, len, st);
      apply_A<double>(P, P->f64, P->plan_A, va, vc, nullptr);
      WC4D_CUDA(cudaMemsetAsync(vc + off3, 0, sizeof(double) * len, st));
      apply_P<double>(P, WC4D_PRECOND_PD, P->f64, vc, va, nullptr);
      WC4D_CUDA(cudaMemsetAsync(va + off3, 0, sizeof(double) * len, st));
      apply_A<double>(P, P->f64, P->plan_A, va, vc, nullptr);
      launch_copy_d(out, vc + off3, len, st);
    };
    // residual-loss value and gradient of sample b of a batch (yb, fb, tb: its rows):
    // loss |S d|^2 / rn2, d = yn + f - tn; gradient 2 S S d / (rn2 nb) into gb
    auto resid_sample = [&](const float* yb, const float* fb, const float* tb, double rn, int nb, float* gb,
                            double* loss_out) {
      net_resid(yb, fb, tb, dd, len, st);
      applyS(dd, sd);
      dot_partial<double>(sd, sd, len, part, nullptr, st);
      dot_finish(part, loss_out, 0, st);
      if (gb) {
        applyS(sd, ssd);
        vec_convert<float, double>(ssd, gb, len, 2.0 / (rn * nb), st);
      }
    };
    // training buffers
    const int B = o.batch;
    const int Hm = std::max(C, sh.H);
    float* params = (float*)dalloc(sizeof(float) * sh.nparams());
    float* grads = (float*)dalloc(sizeof(float) * sh.nparams());
    float* am = (float*)dalloc(sizeof(float) * sh.nparams());
    float* av = (float*)dalloc(sizeof(float) * sh.nparams());
    float* xb = (float*)dalloc(sizeof(float) * B * len);
    float* tb = (float*)dalloc(sizeof(float) * B * len);
    float* outb = (float*)dalloc(sizeof(float) * B * len);
    float* gout = (float*)dalloc(sizeof(float) * B * len);
    float* acts[3];
    for (int l = 0; l < 3; ++l) acts[l] = (float*)dalloc(sizeof(float) * B * (int64_t)Hm * s);
    float* sc0 = (float*)dalloc(sizeof(float) * B * (int64_t)Hm * s);
    float* sc1 = (float*)dalloc(sizeof(float) * B * (int64_t)Hm * s);
    const int64_t wcap = net_wpart_elems(sh, B);
    float* wpart = (float*)dalloc(sizeof(float) * wcap);
    int* d_idx = (int*)dalloc(sizeof(int) * B);
    double* d_loss = (double*)dalloc(sizeof(double));
    std::vector<float> w0 = net_init(sh, o.seed);
    WC4D_CUDA(cudaMemcpy(params, w0.data(), sizeof(float) * w0.size(), cudaMemcpyHostToDevice));
    WC4D_CUDA(cudaMemsetAsync(am, 0, sizeof(float) * sh.nparams(), st));
    WC4D_CUDA(cudaMemsetAsync(av, 0, sizeof(float) * sh.nparams(), st));
    std::mt19937_64 rng(o.seed);
    std::vector<int> order(ntr), idx(B);
    for (int i = 0; i < ntr; ++i) order[i] = i;
    double loss_first = 0, loss_last = 0;
    int step = 0;
    for (int ep = 0; ep < o.epochs; ++ep) {
      std::shuffle(order.begin(), order.end(), rng);
      WC4D_CUDA(cudaMemsetAsync(d_loss, 0, sizeof(double), st));
      int seen = 0;
      for (int b0 = 0; b0 + B <= ntr || (b0 < ntr && b0 == 0); b0 += B) {
        const int nb = std::min(B, ntr - b0);
        for (int b = 0; b < nb; ++b) idx[b] = order[b0 + b];
        WC4D_CUDA(cudaMemcpy(d_idx, idx.data(), sizeof(int) * nb, cudaMemcpyHostToDevice));
        net_gather(yn, d_idx, nb, len, xb, st);
        net_gather(tn, d_idx, nb, len, tb, st);
        net_forward(sh, params, nb, xb, acts, outb, st);
        if (resid_loss) {
          for (int b = 0; b < nb; ++b)
            resid_sample(xb + (int64_t)b * len, outb + (int64_t)b * len, tb + (int64_t)b * len, rn2[idx[b]], nb,
                         gout + (int64_t)b * len, lossv + b);
          std::vector<double> hl(nb);
          WC4D_CUDA(cudaMemcpy(hl.data(), lossv, sizeof(double) * nb, cudaMemcpyDeviceToHost));
          double add = 0;
          for (int b = 0; b < nb; ++b) add += hl[b] / rn2[idx[b]];
          double cur = 0;
          WC4D_CUDA(cudaMemcpy(&cur, d_loss, sizeof(double), cudaMemcpyDeviceToHost));
          cur += add;
          WC4D_CUDA(cudaMemcpy(d_loss, &cur, sizeof(double), cudaMemcpyHostToDevice));
        } else {
          net_loss_grad(sh, nb, xb, outb, tb, tn2, d_idx, gout, d_loss, st);
        }
        net_backward(sh, params, nb, xb, acts, gout, grads, sc0, sc1, wpart, wcap, st);
        net_adam(params, grads, am, av, sh.nparams(), (float)o.lr, ++step, st);
        seen += nb;
      }
      double h = 0;
      WC4D_CUDA(cudaMemcpy(&h, d_loss, sizeof(double), cudaMemcpyDeviceToHost));
      const double mean = h / std::max(1, seen);
      if (ep == 0) loss_first = mean;
      loss_last = mean;
    }
    // the net is kept only if it beats the plain block on the held-out pairs, in the loss's metric
    double el = 0, ep_ = 0;
    if (!resid_loss) {
      el = net_val_error(P, sh, params, yn, tn, tn2, ntr, o.pairs, B, xb, acts, outb, tb, d_idx, d_loss, true);
      ep_ = net_val_error(P, sh, params, yn, tn, tn2, ntr, o.pairs, B, xb, acts, outb, tb, d_idx, d_loss, false);
    } else {
      for (int i = ntr; i < o.pairs; ++i) {
        const float* yi = yn + (int64_t)i * len;
        const float* ti = tn + (int64_t)i * len;
        net_forward(sh, params, 1, yi, acts, outb, st);
        resid_sample(yi, outb, ti, rn2[i], 1, nullptr, lossv);
        resid_sample(yi, nullptr, ti, rn2[i], 1, nullptr, lossv + 1);
        double hl[2];
        WC4D_CUDA(cudaMemcpy(hl, lossv, sizeof(double) * 2, cudaMemcpyDeviceToHost));
        el += hl[0] / rn2[i];
        ep_ += hl[1] / rn2[i];
      }
      el /= nval;
      ep_ /= nval;
    }
    const auto t2 = std::chrono::steady_clock::now();
    std::vector<float> w((size_t)sh.nparams());
    WC4D_CUDA(cudaMemcpy(w.data(), params, sizeof(float) * w.size(), cudaMemcpyDeviceToHost));
    const bool keep = std::sqrt(el) < std::sqrt(ep_);
    P->net_sh = sh;
    WC4D_CUDA(cudaMemcpy(P->net_params, params, sizeof(float) * w.size(), cudaMemcpyDeviceToDevice));
    P->net_on = keep;
    if (ckpt_path) save_net(ckpt_path, sh, w, std::sqrt(el), std::sqrt(ep_));
    if (rep) {
      rep->loss_first = loss_first;
      rep->loss_last = loss_last;
      rep->val_err_learned = std::sqrt(el);
      rep->val_err_plain = std::sqrt(ep_);
      rep->kept = keep ? 1 : 0;
      rep->pairs_train = ntr;
      rep->gen_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
      rep->train_ms = std::chrono::duration<double, std::milli>(t2 - t1).count();
    }
  } catch (...) {
    cudaStreamSynchronize(st);
    for (void* p : owned) cudaFree(p);
    P->net_on = was_on;
    throw;
  }
  WC4D_CUDA(cudaStreamSynchronize(st));
  for (void* p : owned) cudaFree(p);
  return WC4D_OK;
  WC4D_API_END
}

int wc4d_net_grad(int32_t C, int32_t hidden, int32_t s, int32_t B, const float* params, const float* yn,
                  const float* tn, double* loss, float* grads) {
  WC4D_API_BEGIN
  WC4D_CHECK(params && yn && tn && loss && grads, WC4D_ERR_ARG, "null argument");
  WC4D_CHECK(C >= 1 && C <= 64 && hidden >= 1 && hidden <= 64 && s >= 1 && B >= 1 && B <= 4096, WC4D_ERR_ARG,
             "bad network sizes");
  const NetShape sh{C, hidden, s};
  const int64_t len = (int64_t)C * s, np = sh.nparams(), Hm = std::max(C, hidden);
  cudaStream_t st = nullptr;
  std::vector<void*> owned;
  auto dalloc = [&](size_t bytes) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) throw wc4d::Error{WC4D_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e)};
    owned.push_back(p);
    return p;
  };
  try {
    float* dp = (float*)dalloc(sizeof(float) * np);
    float* dg = (float*)dalloc(sizeof(float) * np);
    float* dy = (float*)dalloc(sizeof(float) * B * len);
    float* dt = (float*)dalloc(sizeof(float) * B * len);
    float* out = (float*)dalloc(sizeof(float) * B * len);
    float* gout = (float*)dalloc(sizeof(float) * B * len);
    float* acts[3];
    for (int l = 0; l < 3; ++l) acts[l] = (float*)dalloc(sizeof(float) * B * Hm * s);
    float* sc0 = (float*)dalloc(sizeof(float) * B * Hm * s);
    float* sc1 = (float*)dalloc(sizeof(float) * B * Hm * s);
    const int64_t wcap = net_wpart_elems(sh, B);
    float* wpart = (float*)dalloc(sizeof(float) * wcap);
    double* tn2 = (double*)dalloc(sizeof(double) * B);
    double* dl = (double*)dalloc(sizeof(double));
    WC4D_CUDA(cudaMemcpy(dp, params, sizeof(float) * np, cudaMemcpyHostToDevice));
    WC4D_CUDA(cudaMemcpy(dy, yn, sizeof(float) * B * len, cudaMemcpyHostToDevice));
    WC4D_CUDA(cudaMemcpy(dt, tn, sizeof(float) * B * len, cudaMemcpyHostToDevice));
    std::vector<double> h2(B, 0.0);
    for (int b = 0; b < B; ++b)
      for (int64_t e = 0; e < len; ++e) h2[b] += (double)tn[b * len + e] * tn[b * len + e];
    WC4D_CUDA(cudaMemcpy(tn2, h2.data(), sizeof(double) * B, cudaMemcpyHostToDevice));
    WC4D_CUDA(cudaMemset(dl, 0, sizeof(double)));
    net_forward(sh, dp, B, dy, acts, out, st);
    net_loss_grad(sh, B, dy, out, dt, tn2, nullptr, gout, dl, st);
    net_backward(sh, dp, B, dy, acts, gout, dg, sc0, sc1, wpart, wcap, st);
    WC4D_CUDA(cudaMemcpy(grads, dg, sizeof(float) * np, cudaMemcpyDeviceToHost));
    double h = 0;
    WC4D_CUDA(cudaMemcpy(&h, dl, sizeof(double), cudaMemcpyDeviceToHost));
    *loss = h / B;
  } catch (...) {
    cudaDeviceSynchronize();
    for (void* p : owned) cudaFree(p);
    throw;
  }
  for (void* p : owned) cudaFree(p);
  return WC4D_OK;
  WC4D_API_END
}

// Batched solve of independent windows: a pool of host workers, each with its
// own non-blocking CUDA stream, takes windows largest-first (longest
// processing time first) and runs the window's own solver on its stream, so
// the kernels of small windows overlap on the GPU while other workers wait on
// their convergence polls.
int wc4d_solve_batch(wc4d_problem* const* probs, int32_t count, const double* const* rhs, double* const* x,
                     int32_t use_x0, int32_t mem_kind, int32_t workers, wc4d_info* infos) {
  WC4D_API_BEGIN
  WC4D_CHECK(count >= 0, WC4D_ERR_ARG, "count must be >= 0");
  if (count == 0) return WC4D_OK;
  WC4D_CHECK(probs && rhs && x, WC4D_ERR_ARG, "null argument");
  WC4D_CHECK(mem_kind == WC4D_MEM_HOST || mem_kind == WC4D_MEM_DEVICE, WC4D_ERR_ARG, "bad mem_kind");
  WC4D_CHECK(workers >= 0 && workers <= 64, WC4D_ERR_ARG, "workers must lie in [0, 64]");
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) {
    WC4D_CHECK(probs[i] && rhs[i] && x[i], WC4D_ERR_ARG, "null problem, rhs or x in the batch");
    for (int k = 0; k < i; ++k) WC4D_CHECK(probs[k] != probs[i], WC4D_ERR_ARG, "a problem appears twice in the batch");
    order[i] = i;
  }
  auto cost = [&](int i) {
    const wc4d_problem* P = probs[i];
    return ((double)P->s * P->s + (double)P->p * P->p) * (P->N + 1);
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
  const int nw = workers > 0 ? std::min<int>(workers, count) : std::min(count, 8);
  int dev = 0;
  WC4D_CUDA(cudaGetDevice(&dev));
  for (int i = 0; i < count; ++i) WC4D_CUDA(cudaStreamSynchronize(probs[i]->st));
  std::atomic<int> next{0};
  std::vector<int> status(count, WC4D_OK);
  std::vector<std::string> msg(count);
  std::vector<wc4d_info> loc(count);
  auto work = [&]() {
    cudaStream_t ws = nullptr;
    if (cudaSetDevice(dev) != cudaSuccess || cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) {
      for (int k = next++; k < count; k = next++) {
        status[order[k]] = WC4D_ERR_CUDA;
        msg[order[k]] = "worker stream creation failed";
      }
      return;
    }
    for (int k = next++; k < count; k = next++) {
      const int i = order[k];
      wc4d_problem* P = probs[i];
      cudaStream_t own = P->st;
      P->st = ws;
      status[i] = wc4d_solve(P, rhs[i], x[i], use_x0, mem_kind, &loc[i]);
      if (status[i] != WC4D_OK) msg[i] = wc4d_last_error();
      P->st = own;
    }
    cudaStreamDestroy(ws);
  };
  std::vector<std::thread> pool;
  for (int w = 0; w < nw; ++w) pool.emplace_back(work);
  for (auto& th : pool) th.join();
  if (infos)
    for (int i = 0; i < count; ++i) infos[i] = loc[i];
  for (int i = 0; i < count; ++i)
    if (status[i] != WC4D_OK) {
      wc4d::set_error("window " + std::to_string(i) + ": " + msg[i]);
      return status[i];
    }
  return WC4D_OK;
  WC4D_API_END
}

int wc4d_apply_fp32(wc4d_problem* P, int32_t which, const float* v, float* out) {
  WC4D_API_BEGIN
  WC4D_CHECK(P && v && out, WC4D_ERR_ARG, "null argument");
  WC4D_CHECK(P->o.precision == WC4D_PREC_MIXED || P->o.precision == WC4D_PREC_DF32_P32, WC4D_ERR_ARG,
             "FP32 operators need precision = MIXED or DF32_P32 at setup");
  WC4D_CHECK(which >= 0 && which <= 2, WC4D_ERR_ARG, "which must be 0 (A), 1 (P_D) or 2 (P_I)");
  WC4D_CHECK(which != 1 || P->have_pd, WC4D_ERR_ARG, "P_D needs a problem set up with precond = PD");
  if (which == 0)
    apply_A<float>(P, P->f32, P->plan_A, v, out, nullptr);
  else
    apply_P<float>(P, which - 1, P->f32, v, out, nullptr);
  return WC4D_OK;
  WC4D_API_END
}

int wc4d_synthesize_rhs(wc4d_problem* P, const double* z_b, const double* z_r, int32_t mem_kind, double* rhs) {
  WC4D_API_BEGIN
  WC4D_CHECK(P && z_b && z_r && rhs, WC4D_ERR_ARG, "null argument");
  WC4D_CHECK(mem_kind == WC4D_MEM_HOST || mem_kind == WC4D_MEM_DEVICE, WC4D_ERR_ARG, "bad mem_kind");
  wc4d::synthesize_rhs(P, z_b, z_r, mem_kind, rhs);
  return WC4D_OK;
  WC4D_API_END
}

int wc4d_l96_gauss_newton(wc4d_problem* P, const wc4d_l96_params* prm, const double* xb, const double* y,
                          double* traj, int32_t init_background, int32_t mem_kind, wc4d_info* loop_info) {
  WC4D_API_BEGIN
  WC4D_CHECK(P && xb && y && traj, WC4D_ERR_ARG, "null argument");
  WC4D_CHECK(mem_kind == WC4D_MEM_HOST || mem_kind == WC4D_MEM_DEVICE, WC4D_ERR_ARG, "bad mem_kind");
  const int rc = wc4d::l96_gauss_newton(P, prm, xb, y, traj, init_background != 0, mem_kind, loop_info);
  if (rc != WC4D_OK) wc4d::set_error("an inner solve of the Gauss-Newton loop failed");
  return rc;
  WC4D_API_END
}

int wc4d_l96_linearize(wc4d_problem* P, const wc4d_l96_params* prm, const double* xb, const double* y,
                       const double* traj, int32_t mem_kind, double* rhs) {
  WC4D_API_BEGIN
  WC4D_CHECK(P && xb && y && traj && rhs, WC4D_ERR_ARG, "null argument");
  WC4D_CHECK(mem_kind == WC4D_MEM_HOST || mem_kind == WC4D_MEM_DEVICE, WC4D_ERR_ARG, "bad mem_kind");
  wc4d::l96_linearize(P, prm, xb, y, traj, mem_kind, rhs);
  return WC4D_OK;
  WC4D_API_END
}

int wc4d_problem_dims(const wc4d_problem* P, int64_t* n, int32_t* s, int32_t* N, int32_t* p) {
  if (!P) return WC4D_ERR_ARG;
  if (n) *n = P->n;
  if (s) *s = P->s;
  if (N) *N = P->N;
  if (p) *p = P->p;
  return WC4D_OK;
}

int wc4d_get_matrix(wc4d_problem* P, int32_t which, double* dst) {
  WC4D_API_BEGIN
  WC4D_CHECK(P && dst, WC4D_ERR_ARG, "null argument");
  const double* src = nullptr;
  int64_t cnt = 0;
  switch (which) {
    case 0: src = P->f64.B; cnt = (int64_t)P->s * P->s; break;  // NULL for banded B, Q (refused below)
    case 1: src = P->f64.Q; cnt = (int64_t)P->s * P->s; break;
    case 2:
      src = P->pertime ? P->ptR : P->f64.R;
      cnt = P->pertime ? P->pt_elems : (int64_t)P->p * P->p;
      break;
    case 3:
      src = P->pertime ? P->ptRh : P->d_Rhat;
      cnt = P->pertime ? P->pt_elems : (int64_t)P->p * P->p;
      break;
    default: throw wc4d::Error{WC4D_ERR_ARG, "which must be 0..3"};
  }
  WC4D_CHECK(src != nullptr, WC4D_ERR_ARG, "this problem keeps no dense copy of that matrix (banded B, Q)");
  WC4D_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, P->st));
  WC4D_CUDA(cudaStreamSynchronize(P->st));
  return WC4D_OK;
  WC4D_API_END
}

double wc4d_rhat_param(const wc4d_problem* P) { return P ? P->rhat_param : 0.0; }

void wc4d_destroy(wc4d_problem* P) {
  if (!P) return;
  cudaStreamSynchronize(P->st);
  delete P;
}

const char* wc4d_last_error(void) { return wc4d::g_last_error.c_str(); }

}  // extern "C"
