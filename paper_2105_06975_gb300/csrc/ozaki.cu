// Ozaki-scheme covariance products on the tensor cores (tcgen05, sm_100+).
//
// A product y = op(At) X in the TN form of the stream-K GEMM (k contiguous in
// both operands) is evaluated as a sum of exact BF16 digit products.  Every
// row i of op(At) and every column c of X is cut below a power-of-two scale
// (2^E above the row / column maximum, E from the largest exponent) into an
// integer F < 2^47 (47 bits), written as seven balanced base-128 digits:
//   a_ik = sigma_i sum_t D_t 2^(-5-7t),   x_kc = tau_c sum_u E_u 2^(-5-7u),
// t, u = 0..6 (t = 0 most significant), |D|, |E| <= 64, each exact in BF16.
// (F + 64 sum_j 128^j < 2^49 keeps the balanced digits within seven 7-bit
// fields; with 48 bits a magnitude within 0.8 % of the scale would carry out.)
// The digit products of significance level l = t + u <= 6 (28 of the 49) are
// accumulated in FP32 in tensor memory, one accumulator per level.  A level
// has at most 7 digit pairs, a segment at most 512 k and |D E| <= 2^12, so
// every partial sum is an integer below 2^24 and the accumulation is exact.
// The epilogue combines the seven levels in double-float and scales by
// sigma_i tau_c 2^-10.  The truncation of each operand (2^-47 of its row or
// column maximum) and the dropped levels 7..12 bound the error of an output by
// about 2^-44 K max_k|a_ik| max_k|x_kc|.  (Error-free splitting of a matrix
// product into products that a lower precision evaluates exactly: Ozaki,
// Ogita, Oishi and Rump, Numer. Algorithms 59, 2012.)
//
// Layout of a digit tile (what one bulk copy moves into shared memory): for a
// block of 16 k, the 7 digit matrices of 128 rows (operator) or 64 columns (X)
// follow each other; each is K-major in 8 x 8 core matrices (8 rows of 16
// bytes), the two k-halves of an 8-row group adjacent (128 bytes apart), the
// 8-row groups 256 bytes apart -- the no-swizzle canonical layout of a
// tcgen05 shared-memory operand.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "common.cuh"
#include "ozaki.cuh"

namespace wc4d {

namespace {

constexpr uint64_t OZ_BIAS = 64ull * (1ull + (1ull << 7) + (1ull << 14) + (1ull << 21) + (1ull << 28) +
                                      (1ull << 35) + (1ull << 42));

__device__ __forceinline__ uint64_t mag_bits(double x) {
  return (uint64_t)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// the seven balanced digits of x below 2^(emax - 1022), emax the largest
// biased exponent of its row / column (integer operations only)
__device__ __forceinline__ void digits7(double x, int emax, int d[OZ_DIGITS]) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  uint64_t F = 0;  // floor(|x| 2^(47 - E)) < 2^47
  if (e != 0 && e != 0x7FF) {
    const int sh = 6 + emax - e;
    if (sh < 64) F = ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) >> sh;
  }
  const uint64_t G = F + OZ_BIAS;  // base-128 digits of G minus 64 are the balanced digits of F
  const bool neg = (b >> 63) != 0;
#pragma unroll
  for (int t = 0; t < OZ_DIGITS; ++t) {
    const int v = (int)((G >> (7 * (OZ_DIGITS - 1 - t))) & 127) - 64;
    d[t] = neg ? -v : v;
  }
}

// 2^(emax - 1022) as a float; NaN marks a row / column with a non-finite entry
__device__ __forceinline__ float scale_of(int emax) {
  if (emax == 0x7FF) return __int_as_float(0x7FC00000);
  const int E = emax - 1022;
  if (E < -126) return 0.f;
  if (E > 127) return __int_as_float(0x7F800000);
  return __int_as_float((E + 127) << 23);
}

__device__ __forceinline__ uint32_t bf16_pair(int lo, int hi) {
  const uint32_t a = __bfloat16_as_ushort(__float2bfloat16_rn((float)lo));
  const uint32_t b = __bfloat16_as_ushort(__float2bfloat16_rn((float)hi));
  return a | (b << 16);
}

__device__ __forceinline__ uint64_t block_max_u64(uint64_t v, uint64_t* red) {
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) red[warp] = v;
  __syncthreads();
  uint64_t m = 0;
  for (int w = 0; w < nw; ++w) m = red[w] > m ? red[w] : m;
  __syncthreads();
  return m;
}

// largest magnitude bit pattern of src[0..n) (8 independent loads in flight per thread)
__device__ __forceinline__ uint64_t max_mag_bits(const double* __restrict__ src, int n) {
  uint64_t mx[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int k0 = threadIdx.x; k0 < n; k0 += 8 * blockDim.x) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = k0 + j * blockDim.x;
      const uint64_t v = (k < n) ? mag_bits(src[k]) : 0ull;
      mx[j] = v > mx[j] ? v : mx[j];
    }
  }
#pragma unroll
  for (int j = 1; j < 8; ++j) mx[0] = mx[j] > mx[0] ? mx[j] : mx[0];
  return mx[0];
}

// The digits of the 8 consecutive entries x[0..8) = k 8g..8g+7 of a row /
// column into its tiles (position r of the tile's 128 (64) rows).
__device__ __forceinline__ void store_group_digits(const double x[8], int g, int emax, uint16_t* tiles,
                                                   int64_t tile_elems, int r) {
  const int k0 = 8 * g, kb = k0 >> 4, kh = (k0 >> 3) & 1;
  int dg[8][OZ_DIGITS];
#pragma unroll
  for (int q = 0; q < 8; ++q) digits7(x[q], emax, dg[q]);
  uint16_t* base = tiles + (int64_t)kb * OZ_DIGITS * tile_elems + (r >> 3) * 128 + kh * 64 + (r & 7) * 8;
#pragma unroll
  for (int t = 0; t < OZ_DIGITS; ++t) {
    uint4 v;
    v.x = bf16_pair(dg[0][t], dg[1][t]);
    v.y = bf16_pair(dg[2][t], dg[3][t]);
    v.z = bf16_pair(dg[4][t], dg[5][t]);
    v.w = bf16_pair(dg[6][t], dg[7][t]);
    *reinterpret_cast<uint4*>(base + t * tile_elems) = v;
  }
}

// Digits of one row (operator) or column (X) of length kdim, padded to nkb
// blocks of 16, into tile rt/ct at position r of its 128 (64) rows.
// src == nullptr or a padding row writes zero digits.
__device__ __forceinline__ void write_digits(const double* src, int kdim, int nkb, int emax, uint16_t* tiles,
                                             int64_t tile_elems, int r) {
  for (int g = threadIdx.x; g < 2 * nkb; g += blockDim.x) {
    double x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = 8 * g + q;
      x[q] = (src != nullptr && k < kdim) ? src[k] : 0.0;
    }
    store_group_digits(x, g, emax, tiles, tile_elems, r);
  }
}

// one CTA per padded row i of op(At)
__global__ void __launch_bounds__(128) oz_rows_kernel(const double* __restrict__ At, int64_t lda, int m, int kdim,
                                                      int nkb, uint16_t* __restrict__ Ad, float* __restrict__ As) {
  __shared__ uint64_t red[4];
  const int i = blockIdx.x;
  const double* row = (i < m) ? At + (int64_t)i * lda : nullptr;
  uint64_t mx = row ? max_mag_bits(row, kdim) : 0ull;
  mx = block_max_u64(mx, red);
  const int emax = (int)(mx >> 52);
  if (threadIdx.x == 0) As[i] = row ? scale_of(emax) : 0.f;
  const int rt = i / OZ_BM, r = i % OZ_BM;
  write_digits(row, kdim, nkb, emax, Ad + (int64_t)rt * nkb * OZ_DIGITS * OZ_A_TILE, OZ_A_TILE, r);
}

// one CTA per (op, wide column tile, column of the tile), and ceil(kdim / 128)
// per op for the double-float split of its one-column (GEMV) column, one entry
// per thread (the split's FP64 subtraction and conversions run on the FP64
// pipe: one CTA over the whole column was the launch's long pole)
__global__ void __launch_bounds__(128) oz_cols_kernel(OzColJobs jobs) {
  __shared__ uint64_t red[4];
  pdl_wait();
  pdl_trigger();
  int o = 0;
  while (o + 1 < jobs.n && (int)blockIdx.x >= jobs.cta_base[o + 1]) ++o;
  const OzColJob& jb = jobs.j[o];
  const int local = (int)blockIdx.x - jobs.cta_base[o];
  if (local >= jb.wide * OZ_BN) {
    const int k = (local - jb.wide * OZ_BN) * (int)blockDim.x + (int)threadIdx.x;
    if (k < jb.kdim) {
      const double x = jb.X[(int64_t)jb.gemv_col * jb.ldx + k];
      const float h = __double2float_rn(x);
      jb.Xgh[k] = h;
      jb.Xgl[k] = __double2float_rn(x - (double)h);
    }
    return;
  }
  const int ct = local / OZ_BN, cl = local % OZ_BN;
  const int c = ct * OZ_BN + cl;
  const double* col = (c < jb.ncols) ? jb.X + (int64_t)c * jb.ldx : nullptr;
  uint16_t* tiles = jb.Xd + (int64_t)ct * jb.nkb * OZ_DIGITS * OZ_X_TILE;
  const int ngroups = 2 * jb.nkb;
  constexpr int GR = 2;  // groups of 8 entries a thread keeps in registers (k <= 2048 with 128 threads)
  if (ngroups <= GR * (int)blockDim.x) {
    // one read of the column: the maximum and the digits from the same registers
    double x[GR][8];
    uint64_t mx = 0;
#pragma unroll
    for (int gi = 0; gi < GR; ++gi) {
      const int g = threadIdx.x + gi * blockDim.x;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = 8 * g + q;
        x[gi][q] = (col != nullptr && g < ngroups && k < jb.kdim) ? col[k] : 0.0;
        const uint64_t v = mag_bits(x[gi][q]);
        mx = v > mx ? v : mx;
      }
    }
    mx = block_max_u64(mx, red);
    const int emax = (int)(mx >> 52);
    if (threadIdx.x == 0) jb.Xs[c] = col ? scale_of(emax) : 0.f;
#pragma unroll
    for (int gi = 0; gi < GR; ++gi) {
      const int g = threadIdx.x + gi * blockDim.x;
      if (g < ngroups) store_group_digits(x[gi], g, emax, tiles, OZ_X_TILE, cl);
    }
    return;
  }
  uint64_t mx = col ? max_mag_bits(col, jb.kdim) : 0ull;
  mx = block_max_u64(mx, red);
  const int emax = (int)(mx >> 52);
  if (threadIdx.x == 0) jb.Xs[c] = col ? scale_of(emax) : 0.f;
  write_digits(col, jb.kdim, jb.nkb, emax, tiles, OZ_X_TILE, cl);
}

// ----------------------------------------------------------- tcgen05 kernel
constexpr int OZ_STAGES = 5;
constexpr uint32_t OZ_A_BYTES = OZ_DIGITS * OZ_A_TILE * 2;  // 28672
constexpr uint32_t OZ_X_BYTES = OZ_DIGITS * OZ_X_TILE * 2;  // 14336
constexpr uint32_t OZ_STAGE_BYTES = OZ_A_BYTES + OZ_X_BYTES;
constexpr int OZ_SMEM = OZ_STAGES * OZ_STAGE_BYTES;  // 215040
constexpr int OZ_EPI_WARPS = 8;                      // two per TMEM lane quarter (column halves)
constexpr int OZ_THREADS = 32 * (OZ_EPI_WARPS + 2);  // + one copy warp and one MMA warp
constexpr int OZ_COPY_WARP = OZ_EPI_WARPS, OZ_MMA_WARP = OZ_EPI_WARPS + 1;
// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both
// K-major, M = 128; N / 8 goes in at bit 17
constexpr uint32_t OZ_IDESC_MK = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_BM >> 4) << 24);
constexpr unsigned long long OZ_WAIT_NS = 1000000000ull;  // a wait gives up after 1 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// no-swizzle shared-memory matrix descriptor: start, leading (next core matrix
// along k) and stride (next 8-row group) byte offsets, descriptor version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
         ((uint64_t)1 << 46);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// non-blocking probe of the phase (test_wait returns at once)
__device__ __forceinline__ bool mbar_probe(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred q;\nmbarrier.test_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase of the given parity; false after lim ns or once
// another role has given up.  With the default limit the loop uses try_wait,
// which lets the hardware suspend the thread until the phase completes (the
// time is checked every 64 polls); a shorter limit (a test of the failure
// path) polls with test_wait and checks the time on every poll, so that the
// limit, not the suspension, decides.
__device__ __noinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                       unsigned long long lim) {
  if (lim < OZ_WAIT_NS) {
    const unsigned long long t0 = now_ns();
    for (;;) {
      if (mbar_probe(bar, parity)) return true;
      if (*abort_flag || now_ns() - t0 > lim) return false;
    }
  }
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = now_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_test(bar, parity)) return true;
    if ((it & 63) == 0 && (*abort_flag || now_ns() - t0 > lim)) return false;
  }
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void give_up(volatile int* abort_flag, int* err, int code) {
  *abort_flag = 1;
  if (err) atomicCAS(err, 0, code);
}

// 16 consecutive operator entries (hi, lo) from k = kb on: 16-byte loads when
// the row is 16-byte aligned and all 16 lie below k1
__device__ __forceinline__ void load16(const float* __restrict__ h, const float* __restrict__ l, int kb, int k1,
                                       bool vec, float* oh, float* ol) {
  if (vec && kb + 16 <= k1) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 a = *reinterpret_cast<const float4*>(h + kb + 4 * q);
      const float4 b = *reinterpret_cast<const float4*>(l + kb + 4 * q);
      oh[4 * q] = a.x, oh[4 * q + 1] = a.y, oh[4 * q + 2] = a.z, oh[4 * q + 3] = a.w;
      ol[4 * q] = b.x, ol[4 * q + 1] = b.y, ol[4 * q + 2] = b.z, ol[4 * q + 3] = b.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const bool in = kb + q < k1;
      oh[q] = in ? h[kb + q] : 0.f;
      ol[q] = in ? l[kb + q] : 0.f;
    }
  }
}

// Double-float GEMV segment (one output column, k-range <= OZ_GEMV_K = 128),
// run by the epilogue warps: eight lanes per row, each over 16 consecutive k;
// in pass p warp w takes rows 4 R (W p + w) + g + 4 i, i < R (g = lane / 8,
// W = OZ_EPI_WARPS, R = OZ_GEMV_ROWS), so 32 R operand floats per lane are in
// flight.  X comes split (hi, lo) from the digit kernel.
constexpr int OZ_GEMV_ROWS = 2;
static_assert(OZ_BM % (4 * OZ_GEMV_ROWS * OZ_EPI_WARPS) == 0, "GEMV passes must tile the 128 rows");
__device__ void gemv_segment(const GemmOpT<double>& op, const GemmSeg& sg, float2* __restrict__ dst) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 3, j = lane & 7;
  const int kb = sg.k0 + 16 * j;
  const bool vec = (op.lda & 3) == 0;  // the split arrays start 16-byte aligned
  float xh[16], xl[16];
  load16(op.Xh, op.Xl, kb, sg.k1, true, xh, xl);
#pragma unroll 1
  for (int pass = 0; pass < OZ_BM / (4 * OZ_GEMV_ROWS * OZ_EPI_WARPS); ++pass) {
    const int base = 4 * OZ_GEMV_ROWS * (OZ_EPI_WARPS * pass + warp) + g;
    if (!__any_sync(0xffffffffu, sg.row0 + base < op.m)) break;
    float ah[OZ_GEMV_ROWS][16], al[OZ_GEMV_ROWS][16];
#pragma unroll
    for (int i = 0; i < OZ_GEMV_ROWS; ++i) {
      const int row = sg.row0 + base + 4 * i;
      const int rr = min(row, op.m - 1);
      const int kend = row < op.m ? sg.k1 : kb;
      if (op.Th) {
        // symmetric Toeplitz operator: entry (rr, k) is the first row's entry
        // |k - rr|, found at k in copy rr % 4 from offset toff + rr % 4 - rr
        // (a multiple of 4 floats: 16-byte loads)
        const int64_t o = (int64_t)(rr & 3) * op.tstride + op.toff + (rr & 3) - rr;
        load16(op.Th + o, op.Tl + o, kb, kend, true, ah[i], al[i]);
      } else {
        const int64_t o = (int64_t)rr * op.lda;
        load16(op.Ah + o, op.Al + o, kb, kend, vec, ah[i], al[i]);
      }
    }
    // paired accumulators (even k, odd k of the lane's 16): one FFMA2 / FADD2
    // multiply-add serves two entries, half the issue slots of the scalar form
    float2 sv[OZ_GEMV_ROWS], cv[OZ_GEMV_ROWS];
#pragma unroll
    for (int i = 0; i < OZ_GEMV_ROWS; ++i) sv[i] = cv[i] = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 16; q += 2)
#pragma unroll
      for (int i = 0; i < OZ_GEMV_ROWS; ++i)
        df_mac2(sv[i], cv[i], make_float2(ah[i][q], ah[i][q + 1]), make_float2(al[i][q], al[i][q + 1]),
                make_float2(xh[q], xh[q + 1]), make_float2(xl[q], xl[q + 1]));
#pragma unroll
    for (int i = 0; i < OZ_GEMV_ROWS; ++i) {
      float2 ev, od;
      two_sum(sv[i].x, cv[i].x, ev.x, ev.y);
      two_sum(sv[i].y, cv[i].y, od.x, od.y);
      float2 v = df_add(ev, od);
#pragma unroll
      for (int o = 1; o < 8; o <<= 1)
        v = df_add(v, make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)));
      if (j == 0 && sg.row0 + base + 4 * i < op.m) dst[base + 4 * i] = v;
    }
  }
}

// Setup of the Toeplitz one-column products: the bitwise check, and copy g of
// the reflected first row, entry |v - toff - g| at position v (zero beyond the
// row), so that row i's entries k lie at copy i % 4, position toff + i % 4 - i + k.
__global__ void oz_toeplitz_check_kernel(const double* __restrict__ A, int64_t lda, int m, int* flag) {
  for (int i = blockIdx.y; i < m; i += gridDim.y) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
      const int d = i > k ? i - k : k - i;
      if (__double_as_longlong(A[(int64_t)i * lda + k]) != __double_as_longlong(A[d])) atomicExch(flag, 1);
    }
  }
}
// every digit tile (R, K) of the operator (rt row tiles, nkb blocks) against
// the tile of its offset 128 R - 16 K that the product kernel reads instead:
// one CTA per tile, *flag set on any difference
__global__ void __launch_bounds__(256) oz_toeplitz_tiles_check_kernel(const uint16_t* __restrict__ Ad, int rt,
                                                                      int nkb, int* flag) {
  constexpr int QB = OZ_BM / OZ_BK;
  constexpr int W = OZ_DIGITS * OZ_A_TILE / 8;  // 16-byte words per tile
  for (int64_t t = blockIdx.x; t < (int64_t)rt * nkb; t += gridDim.x) {
    const int R = (int)(t / nkb), K = (int)(t % nkb);
    const int64_t rep = K >= QB * R ? (int64_t)(K - QB * R) : (int64_t)(R - K / QB) * nkb + K % QB;
    if (rep == t) continue;
    const uint4* a = reinterpret_cast<const uint4*>(Ad + t * OZ_DIGITS * OZ_A_TILE);
    const uint4* b = reinterpret_cast<const uint4*>(Ad + rep * OZ_DIGITS * OZ_A_TILE);
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
      const uint4 x = a[w], y = b[w];
      if (x.x != y.x || x.y != y.y || x.z != y.z || x.w != y.w) atomicExch(flag, 1);
    }
  }
}
__global__ void oz_toeplitz_rows_kernel(const float* __restrict__ Ah, const float* __restrict__ Al, int m, int toff,
                                        int64_t tstride, float* __restrict__ Th, float* __restrict__ Tl) {
  const int64_t total = 4 * tstride;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int g = (int)(e / tstride);
    const int64_t v = e - g * tstride;
    const int64_t d = v - toff - g >= 0 ? v - toff - g : toff + g - v;
    Th[e] = d < m ? Ah[d] : 0.f;
    Tl[e] = d < m ? Al[d] : 0.f;
  }
}

// FULL: all 7 digits (the digit count is a compile-time constant and the
// drain and MMA loops unroll as before); otherwise ops.ndig leading digits.
template <bool FULL>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    gemm_tc_kernel(GemmOpsT<double> ops, const GemmSeg* __restrict__ segs, const int* __restrict__ seg_start,
                   float2* __restrict__ partial, const int* __restrict__ done, int* ran, int* err) {
  // No pdl_wait here: the operator digit tiles (written at setup) stream in
  // while the preceding X-digit kernel still runs; only what that kernel
  // writes waits for it (the X digit copies in the copy warp, the scales and
  // GEMV operands in the epilogue warps).  Every kernel before the X-digit
  // kernel has completed (it triggers this launch after its own wait), so the
  // convergence flag and the partial buffer are already safe to use.
  pdl_trigger();
  if (done != nullptr && *(volatile const int*)done) return;
  if (ran != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *ran = 1;
  extern __shared__ __align__(1024) unsigned char oz_smem[];
  __shared__ __align__(8) uint64_t full_bar[OZ_STAGES], empty_bar[OZ_STAGES];
  __shared__ __align__(8) uint64_t tfull_bar, tfree_bar, fin_bar;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int sbeg = seg_start[blockIdx.x], send = seg_start[blockIdx.x + 1];
  // the pipeline waits give up after lim; the drains at the end keep the full
  // OZ_WAIT_NS so that no copy or product is in flight when the CTA exits
  const unsigned long long lim = ops.wait_ns ? ops.wait_ns : OZ_WAIT_NS;
  // the leading nd digits of each operand: the first nd tiles of every digit
  // block are copied and the levels 0..nd-1 accumulated (nd = 7: exact to the
  // 47-bit operands; fewer: a reduced-precision product, 7 nd - 1 bits)
  const int nd = FULL ? OZ_DIGITS : ops.ndig;
  const uint32_t a_bytes = (uint32_t)nd * OZ_A_TILE * 2, x_bytes = (uint32_t)nd * OZ_X_TILE * 2;
  if (tid == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&tfull_bar, 1);
    mbar_init(&tfree_bar, 32 * OZ_EPI_WARPS);
    mbar_init(&fin_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    // 7 level accumulators of 64 columns: 448 of the 512 columns (one CTA per SM)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;
  const uint32_t sbase = smem_u32(oz_smem);

  if (warp == OZ_COPY_WARP) {
    // ---- bulk-copy producer: one stage = the 7 operator and 7 X digit tiles of 16 k
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      // the first OZ_STAGES fills: operator tiles at once, their X tiles once
      // the X-digit kernel has finished (before any stage is waited on again)
      bool waited = false;
      uint32_t pend_dst[OZ_STAGES];
      const uint16_t* pend_src[OZ_STAGES];
      auto flush = [&]() {
        pdl_wait();
        for (int f = 0; f < min(it, OZ_STAGES); ++f)
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  pend_dst[f]),
              "l"(pend_src[f]), "r"(x_bytes), "r"(smem_u32(&full_bar[f]))
              : "memory");
        waited = true;
      };
      for (int si = sbeg; si < send && ok; ++si) {
        const GemmSeg sg = segs[si];
        const GemmOpT<double>& op = ops.op[sg.op];
        if (min(sg.colw, op.ncols - sg.col0) < 2) continue;
        const int nkb = (op.kdim + OZ_BK - 1) / OZ_BK;
        const int rtile = sg.row0 / OZ_BM;
        const uint16_t* asrc = op.Ad + (int64_t)rtile * nkb * OZ_DIGITS * OZ_A_TILE;
        const uint16_t* xsrc = op.Xd + (int64_t)(sg.col0 / OZ_BN) * nkb * OZ_DIGITS * OZ_X_TILE;
        for (int kb = sg.k0 / OZ_BK; kb < (sg.k1 + OZ_BK - 1) / OZ_BK; ++kb, ++it) {
          const int s = it % OZ_STAGES;
          if (!waited && it == OZ_STAGES) flush();
          if (it >= OZ_STAGES && !mbar_wait(&empty_bar[s], ((it / OZ_STAGES) - 1) & 1, &abort_flag, lim)) {
            give_up(&abort_flag, err, 1);
            ok = false;
            break;
          }
          const uint32_t dA = sbase + s * OZ_STAGE_BYTES, dX = dA + OZ_A_BYTES;
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&full_bar[s])),
                       "r"(a_bytes + x_bytes)
                       : "memory");
          // a Toeplitz operator's tile (R, kb) is the tile of the same offset
          // 128 R - 16 kb in row tile 0 (kb >= 8 R) or in blocks 0..7 of row
          // tile R - kb / 8 (setup checked every tile against it bitwise)
          constexpr int QB = OZ_BM / OZ_BK;
          const uint16_t* at = !op.toep_tiles ? asrc + (int64_t)kb * OZ_DIGITS * OZ_A_TILE
                               : kb >= QB * rtile
                                   ? op.Ad + (int64_t)(kb - QB * rtile) * OZ_DIGITS * OZ_A_TILE
                                   : op.Ad + ((int64_t)(rtile - kb / QB) * nkb + kb % QB) * OZ_DIGITS * OZ_A_TILE;
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dA),
              "l"(at), "r"(a_bytes), "r"(smem_u32(&full_bar[s]))
              : "memory");
          if (waited) {
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dX),
                "l"(xsrc + (int64_t)kb * OZ_DIGITS * OZ_X_TILE), "r"(x_bytes), "r"(smem_u32(&full_bar[s]))
                : "memory");
          } else {  // it < OZ_STAGES: stage it, issued by flush()
            pend_dst[it] = dX;
            pend_src[it] = xsrc + (int64_t)kb * OZ_DIGITS * OZ_X_TILE;
          }
        }
      }
      if (!waited) flush();  // fewer than OZ_STAGES fills, or a give-up before the first reuse
      // no copy may still be landing when the CTA exits: wait for the last fill
      // of every stage (already complete unless a wait above gave up)
      for (int f = max(0, it - OZ_STAGES); f < it; ++f) {
        uint64_t* b = &full_bar[f % OZ_STAGES];
        const unsigned long long t0 = now_ns();
        while (!mbar_test(b, (f / OZ_STAGES) & 1) && now_ns() - t0 < OZ_WAIT_NS) {
        }
      }
    }
  } else if (warp == OZ_MMA_WARP) {
    // ---- MMA issuer: 28 digit products per 16 k into the 7 level accumulators
    if (lane == 0) {
      int it = 0, nseg = 0;
      bool ok = true;
      for (int si = sbeg; si < send && ok; ++si) {
        const GemmSeg sg = segs[si];
        const GemmOpT<double>& op = ops.op[sg.op];
        if (min(sg.colw, op.ncols - sg.col0) < 2) continue;
        if (nseg > 0 && !mbar_wait(&tfree_bar, (nseg - 1) & 1, &abort_flag, lim)) {
          give_up(&abort_flag, err, 2);
          break;
        }
        tc_fence_after();
        const int kb0 = sg.k0 / OZ_BK;
        for (int kb = kb0; kb < (sg.k1 + OZ_BK - 1) / OZ_BK; ++kb, ++it) {
          const int s = it % OZ_STAGES;
          if (!mbar_wait(&full_bar[s], (it / OZ_STAGES) & 1, &abort_flag, lim)) {
            give_up(&abort_flag, err, 3);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t aA = sbase + s * OZ_STAGE_BYTES, aX = aA + OZ_A_BYTES;
          // For digit t of the operator the X digit tiles u = 0..6-t lie stacked in
          // shared memory and their level accumulators t+u are adjacent in TMEM,
          // so one MMA of N = 64 (7-t) columns (split at N <= 256) does them all:
          // 10 MMAs per 16 k instead of 28, and each operator digit tile is read
          // from shared memory once or twice instead of 7-t times.
#pragma unroll
          for (int t = 0; t < OZ_DIGITS; ++t) {
            if (t >= nd) break;
#pragma unroll
            for (int u0 = 0; u0 < OZ_DIGITS - t; u0 += 4) {
              if (u0 >= nd - t) break;
              const int cnt = min(4, nd - t - u0);
              const uint64_t da = sdesc(aA + t * (OZ_A_TILE * 2));
              const uint64_t db = sdesc(aX + u0 * (OZ_X_TILE * 2));
              const uint32_t idesc = OZ_IDESC_MK | ((uint32_t)((cnt * OZ_BN) >> 3) << 17);
              const uint32_t acc = (kb > kb0 || t > 0) ? 1u : 0u;
              asm volatile(
                  "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
                  "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tbase + (uint32_t)((t + u0) * OZ_BN)),
                  "l"(da), "l"(db), "r"(idesc), "r"(acc));
            }
          }
          tc_commit(&empty_bar[s]);  // the stage is free once these products have read it
        }
        if (!ok) break;
        tc_commit(&tfull_bar);
        ++nseg;
      }
      // every product issued by this thread has completed before TMEM is freed
      tc_commit(&fin_bar);
      const unsigned long long t0 = now_ns();
      while (!mbar_test(&fin_bar, 0) && now_ns() - t0 < OZ_WAIT_NS) {
      }
    }
  } else {
    // ---- epilogue warps: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows of
    // the tile) and columns 32 (w / 4) .. + 31 of every level
    pdl_wait();  // the GEMV operands and the X scales come from the X-digit kernel
    const int quarter = warp & 3, half = warp >> 2;
    int nseg = 0;
    for (int si = sbeg; si < send; ++si) {
      const GemmSeg sg = segs[si];
      const GemmOpT<double>& op = ops.op[sg.op];
      const int ncv = min(sg.colw, op.ncols - sg.col0);
      float2* dst = partial + (int64_t)sg.slot * (OZ_BM * GEMM_BN);
      if (ncv < 2) {
        gemv_segment(op, sg, dst);
        continue;
      }
      if (!mbar_wait(&tfull_bar, nseg & 1, &abort_flag, lim)) {
        give_up(&abort_flag, err, 4);
        break;
      }
      __syncwarp();
      tc_fence_after();
      // once any role has given up, the launch's outputs are invalid (the host
      // reports the error): later segments write nothing (this segment's
      // accumulators are complete, tfull having arrived)
      const bool write_ok = !abort_flag;
      const int r = 32 * quarter + lane, row = sg.row0 + r;
      const bool rin = row < op.m;
      const float sig = rin ? op.As[row] : 0.f;
#pragma unroll 1
      for (int cc = 2 * half; cc < 2 * half + 2; ++cc) {
        uint32_t v[OZ_DIGITS][16];
#pragma unroll
        for (int l = 0; l < OZ_DIGITS; ++l) {
          if (l >= nd) {  // levels the launch does not accumulate (uniform over the warp)
#pragma unroll
            for (int j = 0; j < 16; ++j) v[l][j] = 0u;
            continue;
          }
          const uint32_t ta = tbase + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(l * OZ_BN + cc * 16);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(v[l][0]), "=r"(v[l][1]), "=r"(v[l][2]), "=r"(v[l][3]), "=r"(v[l][4]), "=r"(v[l][5]),
                "=r"(v[l][6]), "=r"(v[l][7]), "=r"(v[l][8]), "=r"(v[l][9]), "=r"(v[l][10]), "=r"(v[l][11]),
                "=r"(v[l][12]), "=r"(v[l][13]), "=r"(v[l][14]), "=r"(v[l][15])
              : "r"(ta));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = cc * 16 + j;
          // sum_l acc_l 2^(-7l) in double-float, smallest level first (each term
          // exact).  Levels 6, 5, 4 (below 2^-4 together, every accumulator being
          // below 2^24) are summed in plain FP32: their rounding, at most 2^-28 in
          // these units, is a sixth of what the dropped levels 7..12 may already
          // contribute (up to about 2^-25.3); levels 3..0 enter through
          // error-free TwoSum steps.
          float h = fmaf(__uint_as_float(v[OZ_DIGITS - 3][j]), 0x1p-28f,
                         fmaf(__uint_as_float(v[OZ_DIGITS - 2][j]), 0x1p-35f,
                              __uint_as_float(v[OZ_DIGITS - 1][j]) * 0x1p-42f)),
                lo = 0.f;
          static_assert(OZ_DIGITS == 7, "the level split above assumes seven levels");
#pragma unroll
          for (int l = OZ_DIGITS - 4; l >= 0; --l) {
            const float tl = __uint_as_float(v[l][j]) * __int_as_float((127 - 7 * l) << 23);
            float s, e;
            two_sum(tl, h, s, e);
            h = s;
            lo += e;
          }
          float hh, ll;
          fast_two_sum(h, lo, hh, ll);
          if (rin && c < ncv && write_ok) {
            const float f = sig * op.Xs[sg.col0 + c] * 0x1p-10f;
            dst[c * OZ_BM + r] = make_float2(hh * f, ll * f);
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&tfree_bar);
      ++nseg;
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase));
}

}  // namespace

int oz_wide_tiles(int ncols) {
  if (ncols < 2) return 0;
  const int full = ncols / OZ_BN, rem = ncols % OZ_BN;
  return full + (rem >= 2 ? 1 : 0);
}

int64_t oz_operator_elems(int m, int kdim) {
  const int64_t rt = (m + OZ_BM - 1) / OZ_BM, nkb = (kdim + OZ_BK - 1) / OZ_BK;
  return rt * nkb * OZ_DIGITS * OZ_A_TILE;
}

int64_t oz_x_elems(int kdim, int ncols) {
  const int64_t nkb = (kdim + OZ_BK - 1) / OZ_BK;
  return (int64_t)oz_wide_tiles(ncols) * nkb * OZ_DIGITS * OZ_X_TILE;
}

void launch_oz_rows(const double* At, int64_t lda, int m, int kdim, uint16_t* Ad, float* As, cudaStream_t st) {
  const int rt = (m + OZ_BM - 1) / OZ_BM, nkb = (kdim + OZ_BK - 1) / OZ_BK;
  if (rt == 0 || nkb == 0) return;
  oz_rows_kernel<<<rt * OZ_BM, 128, 0, st>>>(At, lda, m, kdim, nkb, Ad, As);
  WC4D_LAUNCH_CHECK();
}

void launch_oz_toeplitz(const double* At, int64_t lda, int m, const float* Ah, const float* Al, float* Th,
                        float* Tl, int* flag, cudaStream_t st) {
  if (m <= 0) return;
  const dim3 grid((unsigned)std::min((m + 255) / 256, 8), (unsigned)std::min(m, 1024));
  oz_toeplitz_check_kernel<<<grid, 256, 0, st>>>(At, lda, m, flag);
  WC4D_LAUNCH_CHECK();
  const int64_t total = 4 * oz_toeplitz_stride(m);
  oz_toeplitz_rows_kernel<<<(unsigned)std::min<int64_t>((total + 255) / 256, 1024), 256, 0, st>>>(
      Ah, Al, m, oz_toeplitz_off(m), oz_toeplitz_stride(m), Th, Tl);
  WC4D_LAUNCH_CHECK();
}

void launch_oz_toeplitz_tiles(const uint16_t* Ad, int m, int kdim, int* flag, cudaStream_t st) {
  const int rt = (m + OZ_BM - 1) / OZ_BM, nkb = (kdim + OZ_BK - 1) / OZ_BK;
  if (rt <= 0 || nkb <= 0) return;
  oz_toeplitz_tiles_check_kernel<<<(unsigned)std::min(rt * nkb, 152 * 8), 256, 0, st>>>(Ad, rt, nkb, flag);
  WC4D_LAUNCH_CHECK();
}

void launch_oz_cols(const OzColJobs& jobs, cudaStream_t st) {
  const int ctas = jobs.cta_base[jobs.n];
  if (jobs.n == 0 || ctas == 0) return;
  WC4D_CUDA(launch_pdl(oz_cols_kernel, dim3(ctas), dim3(128), 0, st, jobs));
  WC4D_LAUNCH_CHECK();
}

void launch_gemm_tc(const GemmOpsT<double>& ops, const GemmSeg* segs, const int* seg_start, int nctas,
                    double* partial, const int* done, int* ran, int* err, cudaStream_t st) {
  static std::once_flag once;
  std::call_once(once, [] {
    WC4D_CUDA(cudaFuncSetAttribute(gemm_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
    WC4D_CUDA(cudaFuncSetAttribute(gemm_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
  });
  WC4D_CHECK(ops.ndig >= 1 && ops.ndig <= OZ_DIGITS, WC4D_ERR_ARG, "internal: digit count out of range");
  if (ops.ndig == OZ_DIGITS)
    WC4D_CUDA(launch_pdl(gemm_tc_kernel<true>, dim3(nctas), dim3(OZ_THREADS), OZ_SMEM, st, ops, segs, seg_start,
                         reinterpret_cast<float2*>(partial), done, ran, err));
  else
    WC4D_CUDA(launch_pdl(gemm_tc_kernel<false>, dim3(nctas), dim3(OZ_THREADS), OZ_SMEM, st, ops, segs, seg_start,
                         reinterpret_cast<float2*>(partial), done, ran, err));
  WC4D_LAUNCH_CHECK();
}

static std::atomic<unsigned long long> g_oz_wait_ns{0};
void oz_set_wait_limit(unsigned long long ns) { g_oz_wait_ns.store(ns, std::memory_order_relaxed); }
unsigned long long oz_wait_limit() { return g_oz_wait_ns.load(std::memory_order_relaxed); }

int oz_resident_ctas() {
  // set by whichever host thread (a batched solve's workers) asks first; all compute the same value
  static std::atomic<int> cached{0};
  if (const int c = cached.load(std::memory_order_relaxed)) return c;
  int dev = 0, sms = 0;
  WC4D_CUDA(cudaGetDevice(&dev));
  WC4D_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int c = std::max(1, sms);
  cached.store(c, std::memory_order_relaxed);
  return c;
}

}  // namespace wc4d
