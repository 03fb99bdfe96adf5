// Circulant covariance products by FFT in FP64 (Sec. 6.1: on the periodic
// uniform grid the SOAR B and Q depend on (i - j) mod s only, so they are
// circulant, diagonalised by the DFT: C = F^{-1} diag(lambda) F with lambda
// real because C is symmetric).  C x, C^{-1} x and (C + delta I)^{-1} x are
// then two transforms and a scaling per column instead of an s x s product.
//
// GB300 runs FP64 at 2 DFMA per clock per SM, so one CTA per column would
// leave most SMs idle behind a few long FP64 chains.  Each complex transform
// (two real columns of one operator packed as re + i im: a real spectrum acts
// on both parts separately) is instead split over a cluster of 8 CTAs with the
// four-step factorisation s = 8 Q, n = Q n1 + n2, k = k1 + 8 k2:
//   X[k1 + 8 k2] = sum_n2 w_Q^(n2 k2) w^(n2 k1) sum_n1 w_8^(n1 k1) x[Q n1 + n2]
// Phase 1: CTA c takes n2 in [c Q/8, (c+1) Q/8): 8-point DFTs over n1 in
//          registers, twiddle w^(n2 k1), each result sent to CTA k1's shared
//          memory (distributed shared memory store).
// Phase 2: CTA k1: length-Q decimation-in-frequency FFT in shared memory
//          (natural order in, bit-reversed out), scaling by lambda (stored in
//          the same bit-reversed cluster layout), decimation-in-time inverse
//          FFT (bit-reversed in, natural out), twiddle w^(-n2 k1), each value
//          sent back to the CTA owning n2.
// Phase 3: CTA c: 8-point inverse DFTs over k1, / s, fused epilogue, store.
// Two cluster barriers separate the phases; both exchanges go through
// distributed shared memory, so HBM sees each input column read once and
// each output column written once.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "circulant.cuh"
#include "model_dev.cuh"

namespace cg = cooperative_groups;

namespace wc4d {
namespace {

// Scalar arithmetic of the transforms.  FP64 mode runs them in FP64; the
// double-float modes (DF32, OZAKI) in double-float pairs on the FP32 pipe
// (value = hi + lo, about 48 significant bits, Dekker / Knuth error-free
// steps): GB300 issues one FP64 warp instruction per 16 SM cycles but an FP32
// one per cycle per sub-partition, so the ~20 FP32 instructions of a
// double-float complex operation still cost far less than its FP64 form.
struct ArithF64 {
  using R = double;
  static __device__ __forceinline__ R add(R a, R b) { return a + b; }
  static __device__ __forceinline__ R sub(R a, R b) { return a - b; }
  static __device__ __forceinline__ R mul(R a, R b) { return a * b; }
  static __device__ __forceinline__ R neg(R a) { return -a; }
  static __device__ __forceinline__ R from(double x) { return x; }
  static __device__ __forceinline__ double to(R a) { return a; }
  static __device__ __forceinline__ R zero() { return 0.0; }
  static __device__ __forceinline__ R sqrt_half() { return 0.70710678118654752440; }
};
struct ArithDF {
  using R = float2;
  static __device__ __forceinline__ R add(R a, R b) { return df_add(a, b); }
  static __device__ __forceinline__ R sub(R a, R b) { return df_add(a, df_neg(b)); }
  static __device__ __forceinline__ R mul(R a, R b) { return df_mul(a, b); }
  static __device__ __forceinline__ R neg(R a) { return df_neg(a); }
  static __device__ __forceinline__ R from(double x) { return df_from(x); }
  static __device__ __forceinline__ double to(R a) { return (double)a.x + (double)a.y; }
  static __device__ __forceinline__ R zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ R sqrt_half() { return make_float2(0.70710677f, 1.21016175e-08f); }
};

// a complex value: 16 bytes in both arithmetics
template <class A>
struct Cx {
  typename A::R re, im;
};
template <class A>
__device__ __forceinline__ Cx<A> cadd(Cx<A> a, Cx<A> b) {
  return {A::add(a.re, b.re), A::add(a.im, b.im)};
}
template <class A>
__device__ __forceinline__ Cx<A> csub(Cx<A> a, Cx<A> b) {
  return {A::sub(a.re, b.re), A::sub(a.im, b.im)};
}
template <class A>
__device__ __forceinline__ Cx<A> cmul(Cx<A> a, Cx<A> w) {
  return {A::sub(A::mul(a.re, w.re), A::mul(a.im, w.im)), A::add(A::mul(a.re, w.im), A::mul(a.im, w.re))};
}
template <class A>
__device__ __forceinline__ Cx<A> cmulc(Cx<A> a, Cx<A> w) {  // a * conj(w)
  return {A::add(A::mul(a.re, w.re), A::mul(a.im, w.im)), A::sub(A::mul(a.im, w.re), A::mul(a.re, w.im))};
}

// 8-point DFT in registers, natural order in and out.  SIGN = -1: forward
// (w_8 = exp(-2 pi i / 8)); +1: inverse without the 1/8.  Radix-2
// decimation in frequency, then the bit-reversed result put back in order.
// Multiplication by w_8^(+-1), w_8^(+-2) = -+i and w_8^(+-3) in closed form.
template <class A, int SIGN>
__device__ __forceinline__ void dft8(Cx<A> (&a)[8]) {
  const typename A::R c = A::sqrt_half();
  // stage h = 4: twiddles w_8^j, j = 0..3
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const Cx<A> u = a[j], v = a[j + 4];
    a[j] = cadd(u, v);
    Cx<A> d = csub(u, v);
    if (j == 1) {
      const typename A::R x = (SIGN < 0) ? A::add(d.re, d.im) : A::sub(d.re, d.im);
      const typename A::R y = (SIGN < 0) ? A::sub(d.im, d.re) : A::add(d.im, d.re);
      d = {A::mul(c, x), A::mul(c, y)};
    }
    if (j == 2) d = (SIGN < 0) ? Cx<A>{d.im, A::neg(d.re)} : Cx<A>{A::neg(d.im), d.re};
    if (j == 3) {
      const typename A::R x = (SIGN < 0) ? A::sub(d.im, d.re) : A::neg(A::add(d.re, d.im));
      const typename A::R y = (SIGN < 0) ? A::neg(A::add(d.re, d.im)) : A::sub(d.re, d.im);
      d = {A::mul(c, x), A::mul(c, y)};
    }
    a[j + 4] = d;
  }
  // stage h = 2: twiddles w_8^(2j) = w_4^j, j = 0, 1
#pragma unroll
  for (int b = 0; b < 8; b += 4) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const Cx<A> u = a[b + j], v = a[b + j + 2];
      a[b + j] = cadd(u, v);
      Cx<A> d = csub(u, v);
      if (j == 1) d = (SIGN < 0) ? Cx<A>{d.im, A::neg(d.re)} : Cx<A>{A::neg(d.im), d.re};
      a[b + j + 2] = d;
    }
  }
  // stage h = 1
#pragma unroll
  for (int b = 0; b < 8; b += 2) {
    const Cx<A> u = a[b], v = a[b + 1];
    a[b] = cadd(u, v);
    a[b + 1] = csub(u, v);
  }
  // bit-reversed positions 1 <-> 4, 3 <-> 6
  Cx<A> t = a[1];
  a[1] = a[4];
  a[4] = t;
  t = a[3];
  a[3] = a[6];
  a[6] = t;
}

__device__ __forceinline__ void epilogue_store(const CircJob& J, const ModelDev& md, int s, int r, int c, double y) {
  if (c >= J.ncols) return;
  double val;
  switch (J.mode) {
    case EPI_SADDLE_C1: {
      const int t = c + J.t0;
      double pre = J.v3[(int64_t)t * s + r];
      if (t >= 1) pre -= model_apply<double>(md, t, J.v3 + (int64_t)(t - 1) * s, r);
      val = y + pre;
      break;
    }
    case EPI_SUB_FROM:
      val = J.Y[r + (int64_t)c * J.ldc] - y;
      break;
    case EPI_NEG_STORE:
      val = -y;
      break;
    default:
      val = y;
  }
  J.C[r + (int64_t)c * J.ldc] = val;
  if (J.Ch != nullptr) {
    const float h = (float)val;
    J.Ch[r + (int64_t)c * J.ldc] = h;
    J.Cl[r + (int64_t)c * J.ldc] = (float)(val - (double)h);
  }
}

template <class A>
__device__ __forceinline__ const typename A::R* job_lam(const CircJob& J);
template <>
__device__ __forceinline__ const double* job_lam<ArithF64>(const CircJob& J) {
  return J.lam;
}
template <>
__device__ __forceinline__ const float2* job_lam<ArithDF>(const CircJob& J) {
  return J.lamdf;
}

template <class A>
__global__ void __launch_bounds__(CIRC_THREADS) circ_kernel(CircJobs jobs, int s, const Cx<A>* __restrict__ tw,
                                                            ModelDev md, const int* __restrict__ done, int* ran) {
  using R = typename A::R;
  pdl_wait();
  pdl_trigger();
  // every CTA of a cluster reads the same flag (written by an earlier grid),
  // so a cluster exits as a whole or not at all
  if (done != nullptr && *(volatile const int*)done) return;
  if (ran != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *ran = 1;
  cg::cluster_group cl = cg::this_cluster();
  // distributed shared memory may be written only once every CTA of the
  // cluster runs
  cl.sync();
  const int rank = (int)cl.block_rank();
  const int tr = blockIdx.x / CIRC_P;
  int jb = 0;
  while (jb + 1 < jobs.n && tr >= jobs.tr_base[jb + 1]) ++jb;
  const CircJob& J = jobs.j[jb];
  const int pr = tr - jobs.tr_base[jb];
  const int ca = 2 * pr, cb = 2 * pr + 1;
  const bool hasb = cb < J.ncols;
  const int Q = s / CIRC_P, QP = Q / CIRC_P;
  extern __shared__ __align__(16) unsigned char circ_raw[];
  Cx<A>* buf = reinterpret_cast<Cx<A>*>(circ_raw);  // phase 2 data: Y[rank, n2], n2 < Q
  Cx<A>* buf2 = buf + Q;                             // phase 3 data: V[k1, n2] for this CTA's n2, k1-major
  const double* xa = J.X + (int64_t)ca * J.ldx;
  const double* xb = J.X + (int64_t)(hasb ? cb : ca) * J.ldx;

  // ---- phase 1: 8-point DFTs over n1 for this CTA's n2
  for (int t = threadIdx.x; t < QP; t += blockDim.x) {
    const int n2 = rank * QP + t;
    Cx<A> u[8];
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) {
      const int idx = Q * n1 + n2;
      u[n1] = {A::from(xa[idx]), hasb ? A::from(xb[idx]) : A::zero()};
    }
    dft8<A, -1>(u);
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) {
      const Cx<A> v = (k1 == 0) ? u[0] : cmul(u[k1], tw[n2 * k1]);
      Cx<A>* dst = cl.map_shared_rank(buf, k1);
      dst[n2] = v;
    }
  }
  cl.sync();

  // ---- phase 2: length-Q FFT over n2 (DIF), lambda, inverse FFT (DIT)
  const int half = Q / 2;
  for (int h = half; h >= 1; h >>= 1) {
    const int stride = (Q / (2 * h)) * CIRC_P;  // w_{2h}^j = w^(8 j Q / (2h))
    for (int b = threadIdx.x; b < half; b += blockDim.x) {
      const int j = b & (h - 1);
      const int i = ((b / h) * 2 * h) + j;
      const Cx<A> u = buf[i], v = buf[i + h];
      buf[i] = cadd(u, v);
      buf[i + h] = (j == 0) ? csub(u, v) : cmul(csub(u, v), tw[j * stride]);
    }
    __syncthreads();
  }
  {
    const R* lam = job_lam<A>(J) + (int64_t)rank * Q;
    for (int i = threadIdx.x; i < Q; i += blockDim.x) {
      const R l = lam[i];
      const Cx<A> u = buf[i];
      buf[i] = {A::mul(u.re, l), A::mul(u.im, l)};
    }
  }
  __syncthreads();
  for (int h = 1; h <= half; h <<= 1) {
    const int stride = (Q / (2 * h)) * CIRC_P;
    for (int b = threadIdx.x; b < half; b += blockDim.x) {
      const int j = b & (h - 1);
      const int i = ((b / h) * 2 * h) + j;
      const Cx<A> u = buf[i];
      const Cx<A> v = (j == 0) ? buf[i + h] : cmulc(buf[i + h], tw[j * stride]);
      buf[i] = cadd(u, v);
      buf[i + h] = csub(u, v);
    }
    __syncthreads();
  }
  // twiddle w^(-n2 k1) and send W[rank, n2] to the CTA owning n2
  for (int n2 = threadIdx.x; n2 < Q; n2 += blockDim.x) {
    const Cx<A> v = (rank == 0) ? buf[n2] : cmulc(buf[n2], tw[n2 * rank]);
    Cx<A>* dst = cl.map_shared_rank(buf2, n2 / QP);
    dst[rank * QP + (n2 % QP)] = v;
  }
  cl.sync();

  // ---- phase 3: 8-point inverse DFTs over k1, / s, epilogue
  const double inv_s = 1.0 / (double)s;
  for (int t = threadIdx.x; t < QP; t += blockDim.x) {
    const int n2 = rank * QP + t;
    Cx<A> u[8];
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) u[k1] = buf2[k1 * QP + t];
    dft8<A, 1>(u);
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) {
      const int r = Q * n1 + n2;
      epilogue_store(J, md, s, r, ca, A::to(u[n1].re) * inv_s);
      if (hasb) epilogue_store(J, md, s, r, cb, A::to(u[n1].im) * inv_s);
    }
  }
}

// double -> double-float pairs (twiddle and spectrum tables of the DF kernel)
__global__ void circ_split_kernel(const double* __restrict__ in, float2* __restrict__ out, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double x = in[i];
    const float h = __double2float_rn(x);
    out[i] = make_float2(h, __double2float_rn(x - (double)h));
  }
}

__global__ void circ_twiddle_kernel(double2* tw, int s) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < s; j += gridDim.x * blockDim.x) {
    double sn, cs;
    sincospi(2.0 * (double)j / (double)s, &sn, &cs);
    tw[j] = make_double2(cs, -sn);
  }
}

// double-double sum (hi, lo) += a * b: exact product error by FMA, TwoSum
__device__ __forceinline__ void dd_mac(double& hi, double& lo, double a, double b) {
  const double p = a * b;
  const double pe = fma(a, b, -p);
  const double t = hi + p;
  const double z = t - hi;
  const double e = (hi - (t - z)) + (p - z);
  hi = t;
  lo += e + pe;
}

__device__ __forceinline__ int bitrev(int x, int bits) { return (int)(__brev((unsigned)x) >> (32 - bits)); }

// one warp per frequency k: lambda_k = sum_j col[j] Re(w^(j k))
__global__ void circ_spectrum_kernel(const double* __restrict__ col, int s, const double2* __restrict__ tw,
                                     double shift, int invert, double* __restrict__ lam, int* flag) {
  const int lane = threadIdx.x & 31;
  const int Q = s / CIRC_P;
  const int qbits = __ffs(Q) - 1;
  for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < s; k += (gridDim.x * blockDim.x) >> 5) {
    double hi = 0.0, lo = 0.0;
    for (int j = lane; j < s; j += 32) {
      const int m = (int)(((int64_t)j * k) % s);
      dd_mac(hi, lo, col[j], tw[m].x);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
      const double t = hi + oh;
      const double z = t - hi;
      const double e = (hi - (t - z)) + (oh - z);
      hi = t;
      lo += ol + e;
    }
    if (lane == 0) {
      const double v = (hi + lo) + shift;
      if (!(v > 0.0) || !isfinite(v)) atomicExch(flag, 1);
      const int k1 = k % CIRC_P, k2 = k / CIRC_P;
      lam[(int64_t)k1 * Q + bitrev(k2, qbits)] = invert ? 1.0 / v : v;
    }
  }
}

// Banded circulant product: one CTA per (job, column, tile of BAND_TILE
// outputs); the tile's inputs with a halo of mv on each side (periodic wrap)
// and the taps are staged in shared memory, so each input is read from HBM
// once per tile; each thread forms 4 outputs from the symmetric taps.
__global__ void __launch_bounds__(256) band_kernel(BandJobs jobs, int s, ModelDev md, const int* __restrict__ done,
                                                   int* ran) {
  pdl_wait();
  pdl_trigger();
  if (done != nullptr && *(volatile const int*)done) return;
  if (ran != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *ran = 1;
  extern __shared__ double band_smem[];
  const int tiles = (s + BAND_TILE - 1) / BAND_TILE;
  int b = blockIdx.x, q = 0;
  while (q + 1 < jobs.n && b >= jobs.j[q].ncols * tiles) {
    b -= jobs.j[q].ncols * tiles;
    ++q;
  }
  const BandJob& J = jobs.j[q];
  const int c = b / tiles, j0 = (b % tiles) * BAND_TILE;
  const int mv = J.mv, w = BAND_TILE + 2 * mv;
  double* xs = band_smem;       // x[j0 - mv .. j0 + BAND_TILE + mv)
  double* taps = band_smem + w;  // row[0 .. mv]: the symmetric half
  const double* x = J.X + (int64_t)c * J.ldx;
  for (int i = threadIdx.x; i < w; i += blockDim.x) {
    int g = j0 - mv + i;
    g %= s;
    g += (g < 0) ? s : 0;
    xs[i] = x[g];
  }
  for (int i = threadIdx.x; i <= mv; i += blockDim.x) taps[i] = J.row[mv + i];
  __syncthreads();
  for (int o = threadIdx.x; o < BAND_TILE; o += blockDim.x) {
    const int j = j0 + o;
    if (j >= s) break;
    const double* xc = xs + mv + o;
    double acc = (taps[0] + J.delta) * xc[0];
    for (int i = 1; i <= mv; ++i) acc = fma(taps[i], xc[i] + xc[-i], acc);
    double val;
    switch (J.mode) {
      case EPI_SADDLE_C1: {
        const int t = c + J.t0;
        double pre = J.v3[(int64_t)t * s + j];
        if (t >= 1) pre -= model_apply<double>(md, t, J.v3 + (int64_t)(t - 1) * s, j);
        val = acc + pre;
        break;
      }
      case EPI_SUB_FROM:
        val = J.Y[j + (int64_t)c * J.ldc] - acc;
        break;
      default:
        val = acc;
    }
    J.C[j + (int64_t)c * J.ldc] = val;
    if (J.Ch != nullptr) {
      const float h = (float)val;
      J.Ch[j + (int64_t)c * J.ldc] = h;
      J.Cl[j + (int64_t)c * J.ldc] = (float)(val - (double)h);
    }
  }
}

__device__ __forceinline__ void atomic_min_double(double* addr, double v) {
  // order-preserving for finite doubles: compare as the double values
  unsigned long long* a = reinterpret_cast<unsigned long long*>(addr);
  unsigned long long old = *a, assumed;
  do {
    assumed = old;
    if (__longlong_as_double((long long)assumed) <= v) return;
    old = atomicCAS(a, assumed, (unsigned long long)__double_as_longlong(v));
  } while (old != assumed);
}

__global__ void band_lambda_kernel(const double* __restrict__ row, int mv, int s, double* out) {
  double mn = INFINITY;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < s; k += gridDim.x * blockDim.x) {
    double lam = row[mv];
    for (int i = 1; i <= mv; ++i) {
      // cos(2 pi i k / s) with the angle reduced exactly: (i k) mod s
      const int m = (int)(((int64_t)i * k) % s);
      lam = fma(2.0 * row[mv + i], cospi(2.0 * (double)m / (double)s), lam);
    }
    mn = fmin(mn, lam);
  }
  for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  if ((threadIdx.x & 31) == 0) atomic_min_double(out, mn);
}

// flag = 1 where |A[i + j s] - A[(i - j) mod s]| > tol A[0] (A SPD: its
// diagonal bounds every entry)
__global__ void circ_check_kernel(const double* __restrict__ A, int s, double tol, int* flag) {
  const double lim = tol * fabs(A[0]);
  const int64_t total = (int64_t)s * s;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % s), j = (int)(e / s);
    int d = i - j;
    d += (d < 0) ? s : 0;
    const double a = A[e];
    if (!(fabs(a - A[d]) <= lim)) atomicExch(flag, 1);
  }
}

}  // namespace

void launch_circ_check(const double* A, int s, double tol, int* flag, cudaStream_t st) {
  const int64_t total = (int64_t)s * s;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 8);
  circ_check_kernel<<<blocks, 256, 0, st>>>(A, s, tol, flag);
  WC4D_LAUNCH_CHECK();
}

void launch_band(const BandJobs& jobs, int s, const ModelDev& md, const int* done, cudaStream_t st) {
  if (jobs.n == 0) return;
  const int tiles = (s + BAND_TILE - 1) / BAND_TILE;
  int ctas = 0, mvmax = 0;
  double flops = 0.0, bytes = 0.0;
  for (int q = 0; q < jobs.n; ++q) {
    ctas += jobs.j[q].ncols * tiles;
    mvmax = std::max(mvmax, jobs.j[q].mv);
    flops += 2.0 * (2 * jobs.j[q].mv + 1) * (double)s * jobs.j[q].ncols;
    const int ep = (jobs.j[q].mode == EPI_SADDLE_C1 || jobs.j[q].mode == EPI_SUB_FROM) ? 1 : 0;
    bytes += 8.0 * s * jobs.j[q].ncols * (2 + ep);
  }
  if (ctas == 0) return;
  const size_t smem = sizeof(double) * (BAND_TILE + 2 * mvmax + mvmax + 1);
  WC4D_CHECK(smem <= 48 * 1024, WC4D_ERR_ARG, "internal: band too wide for the product kernel");
  int* ran = prof_enabled() ? prof_begin(PROF_CIRC, flops, st, bytes) : nullptr;
  WC4D_CUDA(launch_pdl(band_kernel, dim3(ctas), dim3(256), smem, st, jobs, s, md, done, ran));
  WC4D_LAUNCH_CHECK();
  if (ran) prof_end(st);
}

void launch_band_lambda_min(const double* row, int mv, int s, double* out, cudaStream_t st) {
  launch_fill_d(out, INFINITY, 1, st);
  const int blocks = std::min((s + 255) / 256, 152 * 4);
  band_lambda_kernel<<<blocks, 256, 0, st>>>(row, mv, s, out);
  WC4D_LAUNCH_CHECK();
}

void launch_circ_twiddles(double2* tw, int s, cudaStream_t st) {
  circ_twiddle_kernel<<<(s + 255) / 256, 256, 0, st>>>(tw, s);
  WC4D_LAUNCH_CHECK();
}

void launch_circ_spectrum(const double* col, int s, const double2* tw, double shift, int invert, double* lam,
                          int* flag, cudaStream_t st) {
  const int warps = 8;
  const int blocks = std::min((s + warps - 1) / warps, 152 * 8);
  circ_spectrum_kernel<<<blocks, 32 * warps, 0, st>>>(col, s, tw, shift, invert, lam, flag);
  WC4D_LAUNCH_CHECK();
}

void launch_circ(const CircJobs& jobs, int s, const double2* tw, const float4* twdf, const ModelDev& md,
                 const int* done, cudaStream_t st) {
  if (jobs.n == 0) return;
  const int transforms = jobs.tr_base[jobs.n];
  if (transforms == 0) return;
  WC4D_CHECK(circ_size_ok(s), WC4D_ERR_ARG, "internal: circulant product of an unsupported size");
  WC4D_CHECK(!jobs.df || twdf != nullptr, WC4D_ERR_ARG, "internal: double-float transform without its tables");
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(transforms * CIRC_P));
  cfg.blockDim = dim3(CIRC_THREADS);
  cfg.dynamicSmemBytes = 16 * 2 * (s / CIRC_P);
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CIRC_P;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  // algorithmic work: 5 s log2 s flops per complex transform, two transforms
  // and the real spectrum scaling (2 flops per entry) per column pair; bytes:
  // every column read and written once, plus the epilogue operands
  int* ran = nullptr;
  if (prof_enabled()) {
    const double lg = std::log2((double)s);
    double bytes = 0.0;
    for (int q = 0; q < jobs.n; ++q) {
      const int ep = (jobs.j[q].mode == EPI_SADDLE_C1 || jobs.j[q].mode == EPI_SUB_FROM) ? 1 : 0;
      bytes += 8.0 * s * jobs.j[q].ncols * (2 + ep);
    }
    ran = prof_begin(PROF_CIRC, transforms * (10.0 * s * lg + 2.0 * s), st, bytes);
  }
  if (jobs.df)
    WC4D_CUDA(cudaLaunchKernelEx(&cfg, circ_kernel<ArithDF>, jobs, s, reinterpret_cast<const Cx<ArithDF>*>(twdf), md,
                                 done, ran));
  else
    WC4D_CUDA(cudaLaunchKernelEx(&cfg, circ_kernel<ArithF64>, jobs, s, reinterpret_cast<const Cx<ArithF64>*>(tw),
                                 md, done, ran));
  WC4D_LAUNCH_CHECK();
  if (ran) prof_end(st);
}

void launch_circ_split(const double* in, float2* out, int n, cudaStream_t st) {
  circ_split_kernel<<<(n + 255) / 256, 256, 0, st>>>(in, out, n);
  WC4D_LAUNCH_CHECK();
}

}  // namespace wc4d
