// wc4d_apply_saddle_noalloc: the saddle-point product A v computed without
// any device allocation.
//
// Some callers cannot call cudaMalloc: a host thread that shares the GPU with a
// framework whose caching allocator already holds nearly all device memory
// (a fresh cudaMalloc fails or forces that framework to release its cache), or
// a latency-critical loop that cannot afford cudaMalloc/cudaFree, which may
// synchronise the whole device.  For them this entry point takes every input
// and output from the caller and keeps the only scratch it needs -- the split-K
// partial tiles of the covariance products and the inverse observation map --
// in one file-scope device array of fixed size (8 MiB), which every GPU that
// loads the library holds until the process exits.
#include <atomic>
#include <algorithm>

#include "common.cuh"
#include "model_dev.cuh"

namespace wc4d {

template <typename T>
void saddle_c3(const ModelDev& md, const T* v1, const T* v2, const int* inv, int p, T* c3, const int* done,
               cudaStream_t st);

namespace {

constexpr int NA_TILE = GEMM_BM * GEMM_BN;                  // doubles per partial tile
constexpr int NA_MAX_TILES = 240;                           // partial tiles kept in the array
constexpr int NA_MAX_S = 131072;                            // grid points the inverse map can hold
constexpr size_t NA_DOUBLES = (size_t)NA_MAX_TILES * NA_TILE + NA_MAX_S / 2;  // 8 MiB in total

// The scratch array.  Host code must not pass its name to a kernel (on the
// host the name is only a stand-in); it uses the device address fetched with
// cudaGetSymbolAddress below.
static __device__ __align__(256) double g_noalloc_scratch[NA_DOUBLES];

struct NaOp {
  const double* At;  // symmetric m x m covariance (its own transpose)
  const double* X;   // m x ncols, column-major
  int m, ncols;
  int row_tiles, col_tiles, col_width, ksplit;
  int slot0;         // first partial tile of this op
};
struct NaOps {
  NaOp op[3];
  int nops;
};

// CTA b -> (op, row tile, column tile, k split); one partial tile per CTA
__global__ void __launch_bounds__(256) na_gemm_kernel(NaOps ops, double* partial) {
  __shared__ double As[GEMM_BK][GEMM_BM + 1];
  __shared__ double Xs[GEMM_BK][GEMM_BN + 1];
  int b = blockIdx.x, o = 0;
  while (o + 1 < ops.nops && b >= ops.op[o + 1].slot0) ++o;
  const NaOp op = ops.op[o];
  int local = b - op.slot0;
  const int split = local % op.ksplit;
  local /= op.ksplit;
  const int ct = local % op.col_tiles, rt = local / op.col_tiles;
  const int row0 = rt * GEMM_BM, col0 = ct * op.col_width;
  const int ncv = min(op.col_width, op.ncols - col0);
  const int kb = (op.m + GEMM_BK - 1) / GEMM_BK;
  const int k0 = (int)((int64_t)kb * split / op.ksplit) * GEMM_BK;
  const int k1 = min(op.m, (int)((int64_t)kb * (split + 1) / op.ksplit) * GEMM_BK);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4] = {};
  for (int k = k0; k < k1; k += GEMM_BK) {
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;
      const int kk = e % GEMM_BK, ii = e / GEMM_BK;
      const int gi = row0 + ii, gk = k + kk;
      As[kk][ii] = (gi < op.m && gk < k1) ? op.At[gk + (int64_t)gi * op.m] : 0.0;
      Xs[kk][ii] = (ii < ncv && gk < k1) ? op.X[gk + (int64_t)(col0 + ii) * op.m] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GEMM_BK; ++kk) {
      double a[4], x[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) x[j] = Xs[kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], x[j], acc[i][j]);
    }
    __syncthreads();
  }
  // every entry of the tile is written (zeros where rows/columns are absent),
  // so nothing in the array has to start at zero
  double* dst = partial + (int64_t)b * NA_TILE;
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) dst[(ty + 16 * j) * GEMM_BM + tx + 16 * i] = acc[i][j];
}

// c1 = D v1 + L v3 (ops 0: B on time 0, 1: Q on times 1..N), c2 = R v2 + H v3 (op 2)
__global__ void na_reduce_kernel(NaOps ops, const double* partial, ModelDev md, const int* obs, const double* v3,
                                 double* c1, double* c2) {
  const int s = md.s, p = ops.op[2].m;
  const int64_t n1 = (int64_t)s * (md.N + 1), n2 = (int64_t)p * (md.N + 1);
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n1 + n2; g += (int64_t)gridDim.x * blockDim.x) {
    int o, r, c, t;
    if (g < n1) {
      t = (int)(g / s);
      r = (int)(g % s);
      o = (t == 0) ? 0 : 1;
      c = (t == 0) ? 0 : t - 1;
    } else {
      const int64_t e = g - n1;
      t = (int)(e / p);
      r = (int)(e % p);
      o = 2;
      c = t;
    }
    const NaOp& op = ops.op[o];
    const int ct = c / op.col_width, rt = r / GEMM_BM;
    const int first = op.slot0 + (rt * op.col_tiles + ct) * op.ksplit;
    const int off = (c % op.col_width) * GEMM_BM + r % GEMM_BM;
    double acc = 0.0;
    for (int q = 0; q < op.ksplit; ++q) acc += partial[(int64_t)(first + q) * NA_TILE + off];
    if (o < 2) {
      double lv = v3[(int64_t)t * s + r];
      if (t >= 1) lv -= model_apply<double>(md, t, v3 + (int64_t)(t - 1) * s, r);
      c1[(int64_t)t * s + r] = acc + lv;
    } else {
      const int j = obs[r];
      c2[(int64_t)t * p + r] = (j >= 0 && j < s) ? acc + v3[(int64_t)t * s + j] : __longlong_as_double(0x7ff8000000000000LL);
    }
  }
}

__global__ void na_inv_map_kernel(const int* obs, int p, int s, int* inv) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < s; j += gridDim.x * blockDim.x) inv[j] = -1;
}
__global__ void na_inv_fill_kernel(const int* obs, int p, int s, int* inv) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < p; r += gridDim.x * blockDim.x) {
    const int j = obs[r];
    if (j >= 0 && j < s) inv[j] = r;  // out-of-range indices are skipped, never written through
  }
}

// device address of the scratch array, looked up once per device; host
// threads making their first call at the same time may both look it up (the
// same address) but never read a half-written pointer
std::atomic<double*> g_scratch_addr[64];

double* scratch_for_current_device() {
  int dev = 0;
  WC4D_CUDA(cudaGetDevice(&dev));
  WC4D_CHECK(dev >= 0 && dev < 64, WC4D_ERR_ARG, "device ordinal out of range");
  if (double* a = g_scratch_addr[dev].load(std::memory_order_relaxed)) return a;
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess)
    throw Error{WC4D_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e)};
  g_scratch_addr[dev].store((double*)ptr, std::memory_order_relaxed);
  return (double*)ptr;
}

void fill_op(NaOp& op, const double* At, const double* X, int m, int ncols) {
  op.At = At;
  op.X = X;
  op.m = m;
  op.ncols = ncols;
  op.row_tiles = (m + GEMM_BM - 1) / GEMM_BM;
  op.col_tiles = std::max(1, (ncols + GEMM_BN - 1) / GEMM_BN);
  op.col_width = std::max(1, (ncols + op.col_tiles - 1) / op.col_tiles);
  op.ksplit = 1;
}

}  // namespace
}  // namespace wc4d

extern "C" int wc4d_apply_saddle_noalloc(int32_t s, int32_t N, int32_t p, const double* stencil,
                                         const int32_t* obs_idx, const double* B, const double* Q, const double* R,
                                         const double* v, double* out, void* cuda_stream) {
  using namespace wc4d;
  try {
    WC4D_CHECK(stencil && obs_idx && B && Q && R && v && out, WC4D_ERR_ARG, "null argument");
    WC4D_CHECK(s >= 2 && N >= 0 && p >= 1 && p <= s, WC4D_ERR_ARG, "need s >= 2, N >= 0, 1 <= p <= s");
    WC4D_CHECK(s <= NA_MAX_S, WC4D_ERR_ARG, "s exceeds the allocation-free limit of 131072 grid points");
    NaOps ops{};
    ops.nops = 3;
    fill_op(ops.op[0], B, v, s, 1);
    fill_op(ops.op[1], Q, v + s, s, N);
    fill_op(ops.op[2], R, v + (int64_t)(N + 1) * s, p, N + 1);
    int tiles = 0;
    for (int o = 0; o < 3; ++o)
      if (ops.op[o].ncols > 0) tiles += ops.op[o].row_tiles * ops.op[o].col_tiles;
    WC4D_CHECK(tiles <= NA_MAX_TILES, WC4D_ERR_ARG,
               "problem too large for the allocation-free scratch (8 MiB): it needs more than 240 partial "
               "64x64 tiles, i.e. ceil(s/64)*(1 + ceil(N/64)) + ceil(p/64)*ceil((N+1)/64) > 240");
    // split k so that the partial tiles fill the array (better SM occupancy)
    const int ksplit = std::max(1, std::min(16, NA_MAX_TILES / std::max(1, tiles)));
    int slot = 0;
    for (int o = 0; o < 3; ++o) {
      ops.op[o].ksplit = std::min(ksplit, std::max(1, (ops.op[o].m + GEMM_BK - 1) / GEMM_BK));
      ops.op[o].slot0 = slot;
      if (ops.op[o].ncols > 0) slot += ops.op[o].row_tiles * ops.op[o].col_tiles * ops.op[o].ksplit;
    }
    // an op without columns (N = 0) owns no CTA: give it an empty slot range
    if (ops.op[1].ncols == 0) ops.op[1].slot0 = ops.op[2].slot0;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    double* scratch = scratch_for_current_device();
    double* partial = scratch;
    int* inv = (int*)(scratch + (size_t)NA_MAX_TILES * NA_TILE);
    ModelDev md{};
    md.kind = WC4D_MODEL_STENCIL3;
    md.s = s;
    md.N = N;
    md.c0 = stencil[0];
    md.c1 = stencil[1];
    md.c2 = stencil[2];
    // the inverse observation map must start at -1 on every call
    na_inv_map_kernel<<<std::min((s + 255) / 256, 1024), 256, 0, st>>>(obs_idx, p, s, inv);
    WC4D_LAUNCH_CHECK();
    na_inv_fill_kernel<<<std::min((p + 255) / 256, 1024), 256, 0, st>>>(obs_idx, p, s, inv);
    WC4D_LAUNCH_CHECK();
    const double* v1 = v;
    const double* v2 = v + (int64_t)(N + 1) * s;
    const double* v3 = v2 + (int64_t)(N + 1) * p;
    double* c1 = out;
    double* c2 = out + (int64_t)(N + 1) * s;
    double* c3 = c2 + (int64_t)(N + 1) * p;
    saddle_c3<double>(md, v1, v2, inv, p, c3, nullptr, st);
    na_gemm_kernel<<<slot, 256, 0, st>>>(ops, partial);
    WC4D_LAUNCH_CHECK();
    const int64_t total = (int64_t)(s + p) * (N + 1);
    na_reduce_kernel<<<(int)std::min<int64_t>((total + 255) / 256, 152 * 8), 256, 0, st>>>(ops, partial, md, obs_idx,
                                                                                            v3, c1, c2);
    WC4D_LAUNCH_CHECK();
    return WC4D_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.code;
  } catch (...) {
    set_error("unknown exception");
    return WC4D_ERR_CUDA;
  }
}
