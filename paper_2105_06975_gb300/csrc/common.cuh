// Internal declarations shared by the wc4d translation units.
#pragma once
#include <memory>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "wc4d.h"

namespace wc4d {

// An NVTX range over a host scope: setup, factorisation, solve and residual
// phases show up as named ranges in Nsight tools (header-only, a no-op when
// no tool is attached)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ------------------------------------------------------------------ errors
struct Error {
  int code;
  std::string msg;
};

void set_error(const std::string& msg);
inline const char* src_name(const char* path) {
  const char* b = path;
  for (const char* q = path; *q; ++q)
    if (*q == '/') b = q + 1;
  return b;
}
#define WC4D_CUDA(call)                                                              \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      throw ::wc4d::Error{WC4D_ERR_CUDA, std::string(#call) + " at " + ::wc4d::src_name(__FILE__) + ":" + \
                                             std::to_string(__LINE__) + ": " + cudaGetErrorString(e_)};     \
  } while (0)
// every kernel launch of the library is followed by this: it counts the
// launch (wc4d_get_stats) and turns a launch error into an exception
void note_launch();
#define WC4D_LAUNCH_CHECK()                \
  do {                                     \
    ::wc4d::note_launch();                 \
    WC4D_CUDA(cudaGetLastError());         \
  } while (0)
// Programmatic dependent launch (the kernels of a GMRES step): each such
// kernel starts with pdl_wait() -- it returns once the preceding grid has
// completed and its writes are visible (immediately for a plain launch) --
// and then pdl_trigger(), which lets the next grid launch and reach its own
// pdl_wait() while this one runs.  Nothing is read before pdl_wait().
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

#define WC4D_CHECK(cond, code, msg)                        \
  do {                                                     \
    if (!(cond)) throw ::wc4d::Error{(code), (msg)};       \
  } while (0)

// sqrt of a sum of squares that rounding may push slightly below zero: negative
// values give 0, NaN stays NaN (fmax(NaN, 0) would return 0 and hide a
// non-finite input from every check downstream)
__device__ __forceinline__ double sqrt_clamped(double v) { return v > 0.0 ? sqrt(v) : (v == v ? 0.0 : v); }

// q = e / m, r = e % m for a grid-stride index: 32-bit arithmetic when the
// whole range fits (a 64-bit division is a long emulated instruction sequence)
__device__ __forceinline__ void idx_divmod(int64_t e, int m, bool fits32, int& q, int& r) {
  if (fits32) {
    const int ee = (int)e;
    q = ee / m;
    r = ee - q * m;
  } else {
    q = (int)(e / m);
    r = (int)(e - (int64_t)q * m);
  }
}

// ------------------------------------------------------ block reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// two block-wide sums at once (sh: two doubles per warp), results in every thread
__device__ __forceinline__ void block_sum2(double& a, double& b, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  __syncthreads();
  if (lane == 0) {
    sh[wid] = a;
    sh[32 + wid] = b;
  }
  __syncthreads();
  double ta = 0.0, tb = 0.0;
  for (int i = 0; i < nw; ++i) {
    ta += sh[i];
    tb += sh[32 + i];
  }
  a = ta;
  b = tb;
}

// block-wide sum, result valid in every thread (sh: one double per warp)
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; ++i) t += sh[i];
  return t;
}

// ------------------------------------------------- double-float arithmetic
// FP64-class products on the FP32 pipe (GB300 runs FP32 FMA at 64x the FP64
// rate).  Operators are stored split, A = Ah + Al (two FP32 values, ~48
// significant bits); vector entries are split on load.  Each multiply-add
// takes the exact product error of Ah*xh from an FMA, adds the cross terms
// Ah*xl + Al*xh (Al*xl, of relative size 2^-48, is dropped), and accumulates
// into an (s, c) pair with Knuth's TwoSum, so the FP32 rounding of the running
// sum is carried exactly into c.  About 13 FP32 instructions per
// multiply-add; relative error of a length-K product ~ sqrt(K) 2^-48.
__device__ __forceinline__ void df_mac(float& s, float& c, float ah, float al, float xh, float xl) {
  const float p = ah * xh;
  float e = fmaf(ah, xh, -p);
  e = fmaf(ah, xl, e);
  e = fmaf(al, xh, e);
  const float t = s + p;
  const float z = t - s;
  const float err = (s - (t - z)) + (p - z);
  s = t;
  c += err + e;
}

// The same multiply-add on two independent accumulators at once with the
// paired FP32 instructions of sm_100+ (FFMA2 / FADD2 / FMUL2 round each lane
// to nearest like their scalar forms, so the error-free steps are unchanged);
// half the issue slots of two scalar df_mac calls.
__device__ __forceinline__ void df_mac2(float2& s, float2& c, float2 ah, float2 al, float2 xh, float2 xl) {
  const float2 p = __fmul2_rn(ah, xh);
  float2 e = __ffma2_rn(ah, xh, make_float2(-p.x, -p.y));
  e = __ffma2_rn(ah, xl, e);
  e = __ffma2_rn(al, xh, e);
  const float2 t = __fadd2_rn(s, p);
  const float2 z = __fadd2_rn(t, make_float2(-s.x, -s.y));
  const float2 tz = __fadd2_rn(t, make_float2(-z.x, -z.y));
  const float2 err = __fadd2_rn(__fadd2_rn(s, make_float2(-tz.x, -tz.y)), __fadd2_rn(p, make_float2(-z.x, -z.y)));
  s = t;
  c = __fadd2_rn(c, __fadd2_rn(err, e));
}

// Double-float arithmetic on (hi, lo) FP32 pairs (Dekker / Knuth error-free
// transformations): sums and products to ~2^-48 relative without the FP64 pipe.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {  // |a| >= |b|
  s = a + b;
  e = b - (s - a);
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  float s, e;
  two_sum(a.x, b.x, s, e);
  e += a.y + b.y;
  float h, l;
  fast_two_sum(s, e, h, l);
  return make_float2(h, l);
}
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  float h, l;
  fast_two_sum(p, e, h, l);
  return make_float2(h, l);
}
// a double as a normalised pair (FP64 pipe: one conversion, one add, one conversion)
__device__ __forceinline__ float2 df_from(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}
// warp-wide sum of double-float accumulators (s, c) as a pair, valid in every lane
__device__ __forceinline__ float2 df_warp_sum(float s, float c) {
  float h, l;
  two_sum(s, c, h, l);
  float2 v = make_float2(h, l);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float2 w = make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
    v = df_add(v, w);
  }
  return v;
}

// ------------------------------------------------------------ model on device
// M_t for t = 1..N (maps time t-1 to t).  STENCIL3: same 3-point periodic
// stencil for all t.  BANDED: bands[(t-1)*s*w + j*w + (o+lo)] = M_t[j][(j+o) mod s].
struct ModelDev {
  int kind;
  int s, N;
  double c0, c1, c2;
  const double* bands;
  int lo, hi;
};

// ------------------------------------------------------- stream-K FP64 GEMM
// One operand product C = op(At) * X with op(v)_i = sum_k At[k + i*lda] v_k
// (the "TN" form: the k index is contiguous in both operands).  Symmetric
// covariances are their own At; a lower-triangular factor W is applied through
// its stored transpose and vice versa.
constexpr int GEMM_BM = 64;
constexpr int GEMM_BN = 64;
constexpr int GEMM_BK = 16;
constexpr int GEMM_MAX_OPS = 4;

enum { TRI_FULL = 0, TRI_LOWER = 1, TRI_UPPER = 2 };  // op(At) lower: k <= i; upper: k >= i

// Ah/Al: the operator split into FP32 high and low parts (At = Ah + Al to
// 48 bits), used by the double-float ("df32") variant of the FP64 product.
template <typename T>
struct GemmOpT {
  const T* At;
  int64_t lda;
  const T* X;
  int64_t ldx;
  int m, kdim, ncols, tri;
  const float* Ah = nullptr;
  const float* Al = nullptr;
  const float* Xh = nullptr;  // X split the same way (one pass per launch)
  const float* Xl = nullptr;
  // Ozaki digit form (tensor-core products): the operator's rows and X's
  // columns as 7 balanced base-128 digits in BF16, pre-tiled for tcgen05, and
  // one power-of-two scale per row / column (ozaki.cu)
  const uint16_t* Ad = nullptr;
  const float* As = nullptr;
  uint16_t* Xd = nullptr;
  float* Xs = nullptr;
  // a symmetric Toeplitz operator's one-column products (ozaki.cu): its split
  // first row in four reflected copies, copy g holding entry |v - toff - g| at
  // position v, so that row i reads its entries at copy (i % 4), offset
  // toff + (i % 4) - i: contiguous, 16-byte aligned.  nullptr: the dense rows.
  const float* Th = nullptr;
  const float* Tl = nullptr;
  int64_t tstride = 0;  // floats per copy (2 toff + 4)
  int toff = 0;         // 4 ceil(kdim / 4)
  // the same operator's digit tiles (ozaki.cu): tile (R, K) equals the tile
  // of the same offset 128 R - 16 K in row tile 0 or in the first 8 blocks of
  // a row tile, so only those (their union: 8 (rows/128 - 1) + kdim/16
  // tiles) are read; 0: every tile from its own place
  int toep_tiles = 0;
};
template <typename T>
struct GemmOpsT {
  GemmOpT<T> op[GEMM_MAX_OPS];
  int nops;
  int df32 = 0;  // T = double only: run the products in double-float on the FP32 pipe
  int tc = 0;    // T = double only: wide tiles by Ozaki digit products on the tensor cores
  int* err = nullptr;  // tc: device flag set if a wait of the kernel gave up
  unsigned long long wait_ns = 0;  // tc: time limit of the pipeline waits (0: the default, 1 s)
  int ndig = 7;                    // tc: leading digits of each operand the products use (1..7)
};
using GemmOp = GemmOpT<double>;
using GemmOps = GemmOpsT<double>;

struct GemmSeg {
  int op, row0, col0, k0, k1, slot, colw;
};

// Epilogue of the split-K reduction, per op.
enum {
  EPI_STORE = 0,      // C = acc
  EPI_SADDLE_C1 = 1,  // C = acc + (L v3) at time t = col + t0
  EPI_SADDLE_C2 = 2,  // C = acc + v3_t[obs[r]]
  EPI_SUB_FROM = 3,   // C = Y - acc
  EPI_NEG_STORE = 4   // C = -acc
};
template <typename T>
struct EpiT {
  int mode;
  T* C;
  int64_t ldc;
  int t0;          // time index of output column 0
  const T* v3;     // EPI_SADDLE_*: x part of the input vector (time-major, s per time)
  const T* Y;      // EPI_SUB_FROM: minuend, same layout as C
  float* Ch = nullptr;  // T = double, optional: the double-float split of C (same layout)
  float* Cl = nullptr;
};
template <typename T>
struct EpisT {
  EpiT<T> e[GEMM_MAX_OPS];
};
using Epi = EpiT<double>;
using Epis = EpisT<double>;

struct OpShape {
  int m, kdim, ncols, tri;
};

// Static schedule for one set of op shapes: CTA c processes segments
// [seg_start[c], seg_start[c+1]); every segment writes one partial tile slot;
// the reduction sums the slots of each output tile in k order.
struct GemmPlan {
  int nops = 0;
  int bm = GEMM_BM;  // rows per output tile (and per partial slot): 128 for the tensor-core plan
  OpShape shape[GEMM_MAX_OPS];
  int nctas = 0;
  int nslots = 0;
  int* d_seg_start = nullptr;
  GemmSeg* d_segs = nullptr;
  int ntiles = 0;
  int tile_base[GEMM_MAX_OPS];
  int col_tiles[GEMM_MAX_OPS];
  int col_width[GEMM_MAX_OPS];
  int* d_tile_start = nullptr;
  int* d_tile_slots = nullptr;
  int64_t total_out = 0;          // sum over ops of m * ncols
  int64_t out_base[GEMM_MAX_OPS];  // prefix of m * ncols
  double flops = 0;               // 2 * useful multiply-adds
  double tc_bytes = 0;            // tensor-core plan: operator digit tiles and GEMV operands read once,
                                  // X digit tiles once per op, partial tiles written
  double tc_mma_flops = 0;        // tensor-core plan: BF16 flops of the issued digit products
  double tc_digit_bytes = 0;      // the part of tc_bytes that is digit tiles (scales with the digits used)
  double alg_bytes = 0;           // each FP64 operator entry (its triangle) read once, X read once, C written
                                  // once: the floor of any product kernel, whatever its operand form
  double alg_op_bytes[GEMM_MAX_OPS] = {};  // the operator part of alg_bytes, per op
  double tc_gemv_op_bytes[GEMM_MAX_OPS] = {};  // tensor-core plan: GEMV operator rows read, per op
  double tc_digit_op_bytes[GEMM_MAX_OPS] = {};  // tensor-core plan: operator digit tiles read, per op
  std::shared_ptr<void> owner;    // keeps the device arrays alive (plans are shared through a cache)
};

// cost model of the schedule: which product kernel the plan will mostly run
enum { COST_FP64 = 0, COST_DF32 = 1, COST_TC = 2 };
void plan_build(GemmPlan& plan, const std::vector<OpShape>& shapes, int max_ctas, int cost_model = COST_FP64);
// persistent CTAs for the stream-K GEMM: SMs x resident CTAs per SM
int gemm_resident_ctas(bool df32);

// Opt-in kernel profile: CUDA events around the timed kernel classes on the
// launching stream; the kernel itself marks whether it did work (launches that
// exit early on a converged solve do not count).
enum { PROF_GEMM = 0, PROF_ORTH = 1, PROF_GEMM32 = 2, PROF_GEMMDF = 3, PROF_GEMMTC = 4, PROF_CIRC = 5,
       PROF_PERTIME = 6, PROF_CLASSES = 7 };
bool prof_enabled();
// returns a device int* the kernel sets to 1 when it runs (nullptr when off)
int* prof_begin(int cls, double work, cudaStream_t st, double work2 = 0.0, double work3 = 0.0,
                double work4 = 0.0);
void prof_end(cudaStream_t st);
void plan_free(GemmPlan& plan);

template <typename T>
void gemm_run(const GemmPlan& plan, const GemmOpsT<T>& ops, const EpisT<T>& epis, T* partial,
              const ModelDev& model, const int* obs, const int* done, cudaStream_t st);

// ---------------------------------------------------------------- kernels
// tab: s doubles of scratch (the correlation by grid distance), stream-ordered
void launch_soar_fill(double* M, int m, const int* idx, int s, double sigma2, double ell, double* tab,
                      cudaStream_t st);
void launch_copy_d(double* dst, const double* src, int64_t n, cudaStream_t st);
void launch_fill_d(double* dst, double v, int64_t n, cudaStream_t st);
void launch_add_diag(double* A, int m, int64_t lda, const double* shift_dev, double shift, cudaStream_t st);
void launch_keep_diag(double* A, int m, cudaStream_t st);
void launch_block_sumsq(const double* A, int m, const int* pst, int nblocks, double* out, cudaStream_t st);
void launch_zero_across_runs(double* A, int m, const int* run, cudaStream_t st);
void launch_transpose(const double* A, double* At, int m, cudaStream_t st);
void launch_symmetrize(double* A, int m, cudaStream_t st);
void launch_to_float(const double* a, float* b, int64_t n, cudaStream_t st);
// hi = fl32(a), lo = fl32(a - hi): a = hi + lo to about 48 bits
void launch_split_df(const double* a, float* hi, float* lo, int64_t n, cudaStream_t st);
// the same for an m x ncols block with leading dimension ld, written densely (ld = m)
struct SplitBlocks {
  const double* a[4];
  int64_t ld[4];
  int m[4];
  int off[5];  // dense offsets of each block; off[n] = total
  int n = 0, total = 0;
};
void launch_split_df_multi(const SplitBlocks& sb, float* hi, float* lo, cudaStream_t st);
void launch_split_df_block(const double* a, int64_t ld, int m, int ncols, float* hi, float* lo, cudaStream_t st);
void launch_inv_map(const int* obs, int p, int* inv, int s, cudaStream_t st);
void launch_check_obs(const int* obs, int p, int s, int* flag, cudaStream_t st);
void launch_check_finite(const double* a, int64_t n, int* flag, cudaStream_t st);

// Cholesky A = L L^T in place (lower), A is m x m col-major; *info = first bad pivot (1-based) or 0.
void cholesky(double* A, int m, int* info, cudaStream_t st, double* scratch);
// W = L^{-1} for lower-triangular L (m x m); Wt = W^T. scratch >= m*64 doubles.
void tri_inverse(const double* L, double* W, double* Wt, int m, cudaStream_t st, double* scratch);
// Symmetric eigen-decomposition by cyclic Jacobi: A (m x m, overwritten by a
// near-diagonal matrix), V eigenvectors (columns).  m even; returns sweeps used.
int jacobi_eigh(double* A, double* V, int m, cudaStream_t st, double* rot, int* d_count, int max_sweeps);
// Rhat builders on device (lam: diag of the Jacobi result)
void launch_rr_shift(const double* Adiag_src, int m, double kappa, double* gamma_out, cudaStream_t st);
void launch_me_scale(const double* Ajac, const double* V, int m, double kappa, double* U, double* T_out,
                     cudaStream_t st);

// Model / time operators
void launch_lhat_sweep(const ModelDev& md, int k, const double* v, double* z, bool transpose, bool identity_model,
                       const int* done, cudaStream_t st);
void launch_saddle_c3(const ModelDev& md, const double* v1, const double* v2, const int* inv, int p, double* c3,
                      const int* done, cudaStream_t st);

}  // namespace wc4d
