// Krylov kernels: MINRES (preconditioned Lanczos form, Elman-Silvester-Wathen
// Ch. 4) and right-preconditioned (F)GMRES with CGS2 Arnoldi.  Dot products use
// a fixed grid of DOT_BLOCKS blocks and warp-shuffle block reductions; the
// partial sums are added in a fixed order by every consumer, so results are
// bitwise reproducible run to run.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>

#include "krylov.cuh"

namespace wc4d {

// sum of DOT_BLOCKS partials in fixed order (whole block cooperates, same result everywhere)
__device__ __forceinline__ double sum_partials(const double* __restrict__ part, double* sh) {
  double v = 0.0;
  for (int i = threadIdx.x; i < DOT_BLOCKS; i += blockDim.x) v += part[i];
  return block_sum(v, sh);
}

template <typename T>
__global__ void __launch_bounds__(DOT_THREADS) dot_partial_kernel(const T* __restrict__ a, const T* __restrict__ b,
                                                                  int64_t n, double* __restrict__ part,
                                                                  const int* done) {
  if (done != nullptr && *(volatile const int*)done) return;
  __shared__ double sh[32];
  double v = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    v += (double)a[e] * (double)b[e];
  v = block_sum(v, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}
template <typename T>
void dot_partial(const T* a, const T* b, int64_t n, double* part, const int* done, cudaStream_t st) {
  dot_partial_kernel<T><<<DOT_BLOCKS, DOT_THREADS, 0, st>>>(a, b, n, part, done);
  WC4D_LAUNCH_CHECK();
}
template void dot_partial<double>(const double*, const double*, int64_t, double*, const int*, cudaStream_t);
template void dot_partial<float>(const float*, const float*, int64_t, double*, const int*, cudaStream_t);

__global__ void dot_finish_kernel(const double* part, double* out, int sqrt_it) {
  __shared__ double sh[32];
  const double v = sum_partials(part, sh);
  if (threadIdx.x == 0) *out = sqrt_it ? sqrt_clamped(v) : v;
}
void dot_finish(const double* part, double* out, int sqrt_it, cudaStream_t st) {
  dot_finish_kernel<<<1, DOT_THREADS, 0, st>>>(part, out, sqrt_it);
  WC4D_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ MINRES
__global__ void minres_init_kernel(const double* part_gamma, double* sc, DevStatus* stat, double tol) {
  __shared__ double sh[32];
  const double g2 = sum_partials(part_gamma, sh);
  if (threadIdx.x == 0) {
    const double g = sqrt_clamped(g2);
    sc[MS_GAMMA] = g;
    sc[MS_GAMMA_OLD] = 1.0;
    sc[MS_ETA] = g;
    sc[MS_ETA0] = g > 0.0 ? g : 1.0;
    sc[MS_C] = 1.0;
    sc[MS_C_OLD] = 1.0;
    sc[MS_S] = 0.0;
    sc[MS_S_OLD] = 0.0;
    stat->done = 0;
    stat->status = 0;
    stat->iters = 0;
    stat->est = 1.0;
    stat->tol_est = tol;
    if (!(g2 >= 0.0) || !isfinite(g2)) {
      stat->done = 1;
      stat->status = isfinite(g2) ? WC4D_ERR_BREAKDOWN : WC4D_ERR_NONFINITE;
    } else if (g == 0.0) {
      stat->done = 1;
      stat->est = 0.0;
    }
  }
}
void minres_init(const double* part_gamma, double* sc, DevStatus* stat, double tol, cudaStream_t st) {
  minres_init_kernel<<<1, DOT_THREADS, 0, st>>>(part_gamma, sc, stat, tol);
  WC4D_LAUNCH_CHECK();
}

// v_new = A z / gamma - (delta/gamma) v - (gamma/gamma_old) v_old with
// delta = <A z, z> / gamma^2  (z is the unscaled P^{-1} v)
__global__ void __launch_bounds__(DOT_THREADS) minres_v_kernel(const double* part_delta, const double* sc,
                                                               const double* __restrict__ Az,
                                                               const double* __restrict__ v,
                                                               const double* __restrict__ v_old,
                                                               double* __restrict__ v_new, int64_t n,
                                                               const int* done) {
  if (done != nullptr && *(volatile const int*)done) return;
  __shared__ double sh[32];
  const double g = sc[MS_GAMMA], go = sc[MS_GAMMA_OLD];
  const double delta = sum_partials(part_delta, sh) / (g * g);
  const double a = 1.0 / g, b = delta / g, c = g / go;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    v_new[e] = a * Az[e] - b * v[e] - c * v_old[e];
}
void minres_v_update(const double* part_delta, const double* sc, const double* Az, const double* v,
                     const double* v_old, double* v_new, int64_t n, const int* done, cudaStream_t st) {
  minres_v_kernel<<<DOT_BLOCKS, DOT_THREADS, 0, st>>>(part_delta, sc, Az, v, v_old, v_new, n, done);
  WC4D_LAUNCH_CHECK();
}

// MINRES scalars of one iteration from the two dot products (identical in
// every block: same inputs, same summation order).
struct MinresStep {
  double g, gn, gn2, delta, c, s, cn, sn, a1, a2, a3, eta;
};
__device__ __forceinline__ MinresStep minres_scalars(const double* part_delta, const double* part_gamma,
                                                     const double* sc, double* sh) {
  MinresStep m;
  m.g = sc[MS_GAMMA];
  m.delta = sum_partials(part_delta, sh) / (m.g * m.g);
  m.gn2 = sum_partials(part_gamma, sh);
  m.gn = sqrt_clamped(m.gn2);
  m.c = sc[MS_C];
  m.s = sc[MS_S];
  m.eta = sc[MS_ETA];
  const double co = sc[MS_C_OLD], so = sc[MS_S_OLD];
  const double a0 = m.c * m.delta - co * m.s * m.g;
  m.a1 = hypot(a0, m.gn);
  m.a2 = m.s * m.delta + co * m.c * m.g;
  m.a3 = so * m.g;
  m.cn = a0 / m.a1;
  m.sn = m.gn / m.a1;
  return m;
}

// w_new = (z/gamma - a3 w_old - a2 w) / a1,  x += c_new eta w_new
__global__ void __launch_bounds__(DOT_THREADS) minres_update_kernel(
    const double* part_delta, const double* part_gamma, const double* sc, const double* __restrict__ z,
    const double* __restrict__ w_old, const double* __restrict__ w, double* __restrict__ w_new, double* __restrict__ x,
    int64_t n, const int* done) {
  if (*(volatile const int*)done) return;
  __shared__ double sh[32];
  const MinresStep m = minres_scalars(part_delta, part_gamma, sc, sh);
  const double ig = 1.0 / m.g, ia1 = 1.0 / m.a1, step = m.cn * m.eta;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double wn = (z[e] * ig - m.a3 * w_old[e] - m.a2 * w[e]) * ia1;
    w_new[e] = wn;
    x[e] += step * wn;
  }
}

// commits the new scalar state and the stopping decision (separate launch, so
// the flag it sets is only seen by later kernels)
__global__ void minres_commit_kernel(const double* part_delta, const double* part_gamma, const double* sc,
                                     double* sc_out, DevStatus* stat) {
  if (*(volatile const int*)&stat->done) return;
  __shared__ double sh[32];
  const MinresStep m = minres_scalars(part_delta, part_gamma, sc, sh);
  if (threadIdx.x != 0) return;
  const double eta_n = -m.sn * m.eta;
  sc_out[MS_GAMMA] = m.gn;
  sc_out[MS_GAMMA_OLD] = m.g;
  sc_out[MS_ETA] = eta_n;
  sc_out[MS_ETA0] = sc[MS_ETA0];
  sc_out[MS_C] = m.cn;
  sc_out[MS_C_OLD] = m.c;
  sc_out[MS_S] = m.sn;
  sc_out[MS_S_OLD] = m.s;
  const double est = fabs(eta_n) / sc[MS_ETA0];
  stat->iters += 1;
  stat->est = est;
  if (!isfinite(est) || !isfinite(m.gn2)) {
    stat->status = WC4D_ERR_NONFINITE;
    stat->done = 1;
  } else if (m.gn2 < 0.0) {
    stat->status = WC4D_ERR_BREAKDOWN;
    stat->done = 1;
  } else if (est <= stat->tol_est || m.gn == 0.0) {
    stat->done = 1;
  }
}

void minres_update(const double* part_delta, const double* part_gamma, const double* sc_in, double* sc_out,
                   const double* z, const double* w_old, const double* w, double* w_new, double* x, int64_t n,
                   DevStatus* stat, cudaStream_t st) {
  minres_update_kernel<<<DOT_BLOCKS, DOT_THREADS, 0, st>>>(part_delta, part_gamma, sc_in, z, w_old, w, w_new, x, n,
                                                           &stat->done);
  WC4D_LAUNCH_CHECK();
  minres_commit_kernel<<<1, DOT_THREADS, 0, st>>>(part_delta, part_gamma, sc_in, sc_out, stat);
  WC4D_LAUNCH_CHECK();
}

// ------------------------------------------------------------------- GMRES
// part[i * nchunks + c] = sum over chunk c (ORTH_CHUNK elements) of V_i . w.
// Grid (chunks, vector groups of ORTH_G): every thread holds ORTH_U elements of
// w and issues ORTH_G x ORTH_U independent loads of the basis, enough bytes in
// flight to stream V at HBM rate.
template <typename T>
__global__ void __launch_bounds__(DOT_THREADS) gm_mdot_kernel(const T* __restrict__ V, int64_t ldv, int cnt,
                                                              const T* __restrict__ w, int64_t n,
                                                              double* __restrict__ part, const int* done,
                                                              int* ran) {
  if (done != nullptr && *(volatile const int*)done) return;
  if (ran != nullptr && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *ran = 1;
  __shared__ double sh[DOT_THREADS / 32][ORTH_G];
  const int chunk = blockIdx.x, i0 = blockIdx.y * ORTH_G;
  const int64_t e0 = (int64_t)chunk * ORTH_CHUNK + threadIdx.x;
  double wv[ORTH_U];
#pragma unroll
  for (int u = 0; u < ORTH_U; ++u) {
    const int64_t e = e0 + (int64_t)u * DOT_THREADS;
    wv[u] = e < n ? (double)w[e] : 0.0;
  }
  double acc[ORTH_G];
#pragma unroll
  for (int g = 0; g < ORTH_G; ++g) {
    acc[g] = 0.0;
    if (i0 + g < cnt) {
      const T* vi = V + (int64_t)(i0 + g) * ldv;
#pragma unroll
      for (int u = 0; u < ORTH_U; ++u) {
        const int64_t e = e0 + (int64_t)u * DOT_THREADS;
        if (e < n) acc[g] += (double)vi[e] * wv[u];
      }
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int g = 0; g < ORTH_G; ++g) {
    const double v = warp_sum(acc[g]);
    if (lane == 0) sh[wid][g] = v;
  }
  __syncthreads();
  if (threadIdx.x < ORTH_G && i0 + threadIdx.x < cnt) {
    double s = 0.0;
    for (int k = 0; k < DOT_THREADS / 32; ++k) s += sh[k][threadIdx.x];
    part[(int64_t)(i0 + threadIdx.x) * gridDim.x + chunk] = s;
  }
}
template <typename T>
void gm_mdot(const T* V, int64_t ldv, int cnt, const T* w, int64_t n, double* part, const int* done,
             cudaStream_t st) {
  int* ran = prof_begin(PROF_ORTH, (double)(cnt + 1) * n * sizeof(T), st);
  dim3 grid(orth_chunks(n), (cnt + ORTH_G - 1) / ORTH_G);
  gm_mdot_kernel<T><<<grid, DOT_THREADS, 0, st>>>(V, ldv, cnt, w, n, part, done, ran);
  WC4D_LAUNCH_CHECK();
  if (ran) prof_end(st);
}
template void gm_mdot<double>(const double*, int64_t, int, const double*, int64_t, double*, const int*, cudaStream_t);
template void gm_mdot<float>(const float*, int64_t, int, const float*, int64_t, double*, const int*, cudaStream_t);

// h[i] = sum over chunks of part[i * nchunks + c], fixed order
__global__ void gm_mdot_reduce_kernel(const double* part, int nchunks, double* h, const int* done) {
  pdl_wait();
  pdl_trigger();
  if (done != nullptr && *(volatile const int*)done) return;
  __shared__ double sh[32];
  const double* p = part + (int64_t)blockIdx.x * nchunks;
  double v = 0.0;
  for (int c = threadIdx.x; c < nchunks; c += blockDim.x) v += p[c];
  v = block_sum(v, sh);
  if (threadIdx.x == 0) h[blockIdx.x] = v;
}
void gm_mdot_reduce(const double* part, int cnt, int nchunks, double* h, const int* done, cudaStream_t st) {
  WC4D_CUDA(launch_pdl(gm_mdot_reduce_kernel, dim3(cnt), dim3(DOT_THREADS), 0, st, part, nchunks, h, done));
  WC4D_LAUNCH_CHECK();
}

// w -= V h over cnt basis vectors, eight independent loads in flight per thread
template <typename T>
__global__ void __launch_bounds__(DOT_THREADS) gm_mupdate_kernel(const T* __restrict__ V, int64_t ldv, int cnt,
                                                                 const double* __restrict__ h, T* __restrict__ w,
                                                                 int64_t n, const int* done, int* ran) {
  if (done != nullptr && *(volatile const int*)done) return;
  if (ran != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *ran = 1;
  extern __shared__ double hs[];
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) hs[i] = h[i];
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int i = 0;
    for (; i + 8 <= cnt; i += 8) {
      const T* p = V + (int64_t)i * ldv + e;
      const double x0 = (double)p[0], x1 = (double)p[ldv], x2 = (double)p[2 * ldv], x3 = (double)p[3 * ldv];
      const double x4 = (double)p[4 * ldv], x5 = (double)p[5 * ldv], x6 = (double)p[6 * ldv], x7 = (double)p[7 * ldv];
      a0 += hs[i] * x0 + hs[i + 4] * x4;
      a1 += hs[i + 1] * x1 + hs[i + 5] * x5;
      a2 += hs[i + 2] * x2 + hs[i + 6] * x6;
      a3 += hs[i + 3] * x3 + hs[i + 7] * x7;
    }
    for (; i < cnt; ++i) a0 += hs[i] * (double)V[(int64_t)i * ldv + e];
    w[e] = (T)((double)w[e] - ((a0 + a1) + (a2 + a3)));
  }
}
template <typename T>
void gm_mupdate(const T* V, int64_t ldv, int cnt, const double* h, T* w, int64_t n, const int* done,
                cudaStream_t st) {
  int* ran = prof_begin(PROF_ORTH, (double)(cnt + 2) * n * sizeof(T), st);
  const int nb = (int)std::min<int64_t>((n + DOT_THREADS - 1) / DOT_THREADS, 152 * 16);
  gm_mupdate_kernel<T><<<nb, DOT_THREADS, sizeof(double) * cnt, st>>>(V, ldv, cnt, h, w, n, done, ran);
  WC4D_LAUNCH_CHECK();
  if (ran) prof_end(st);
}
template void gm_mupdate<double>(const double*, int64_t, int, const double*, double*, int64_t, const int*,
                                 cudaStream_t);
template void gm_mupdate<float>(const float*, int64_t, int, const double*, float*, int64_t, const int*, cudaStream_t);

// v0 = r0 / beta, g = (beta, 0, ...), status reset
template <typename T>
__global__ void gm_init_kernel(const T* __restrict__ r0, const double* part_beta, T* __restrict__ v0, double* g,
                               DevStatus* stat, double tol, int64_t n) {
  __shared__ double sh[32];
  const double beta = sqrt_clamped(sum_partials(part_beta, sh));
  const double ib = beta > 0.0 ? 1.0 / beta : 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    v0[e] = (T)((double)r0[e] * ib);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    g[0] = beta;
    stat->done = (beta == 0.0) ? 1 : 0;
    stat->status = isfinite(beta) ? 0 : WC4D_ERR_NONFINITE;
    if (!isfinite(beta)) stat->done = 1;
    stat->iters = 0;
    stat->est = 1.0;
    stat->tol_est = tol;
  }
}
template <typename T>
void gm_init(const T* r0, const double* part_beta, T* v0, double* g, DevStatus* stat, double tol, int64_t n,
             cudaStream_t st) {
  gm_init_kernel<T><<<DOT_BLOCKS, DOT_THREADS, 0, st>>>(r0, part_beta, v0, g, stat, tol, n);
  WC4D_LAUNCH_CHECK();
}
template void gm_init<double>(const double*, const double*, double*, double*, DevStatus*, double, int64_t,
                              cudaStream_t);
template void gm_init<float>(const float*, const double*, float*, double*, DevStatus*, double, int64_t, cudaStream_t);

// Column j of the Hessenberg matrix, previous Givens rotations, the new one,
// the residual estimate |g_{j+1}| / ||b||.  The column and the rotations are
// staged in shared memory so the serial rotation chain runs at shared-memory
// latency (the chain has j dependent steps).
__global__ void gm_hessenberg_kernel(int j, const double* h1, const double* h2, const double* part_norm, double* H,
                                     int ldh, double* cs, double* sn, double* g, double* hnext, DevStatus* stat,
                                     const double* bnorm) {
  extern __shared__ double sm[];  // col[j+2], c[j], s[j]
  __shared__ double sh[32];
  if (*(volatile const int*)&stat->done) return;
  const double nrm2 = sum_partials(part_norm, sh);
  double* col = sm;
  double* c_ = sm + (j + 2);
  double* s_ = c_ + j;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) col[i] = h1[i] + h2[i];
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    c_[i] = cs[i];
    s_[i] = sn[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double hn = sqrt_clamped(nrm2);
    col[j + 1] = hn;
    *hnext = hn;
    for (int i = 0; i < j; ++i) {
      const double a = col[i], b = col[i + 1];
      col[i] = c_[i] * a + s_[i] * b;
      col[i + 1] = -s_[i] * a + c_[i] * b;
    }
    double c = 1.0, s = 0.0;
    if (col[j + 1] != 0.0) {
      const double r = hypot(col[j], col[j + 1]);
      c = col[j] / r;
      s = col[j + 1] / r;
    }
    cs[j] = c;
    sn[j] = s;
    col[j] = c * col[j] + s * col[j + 1];
    col[j + 1] = 0.0;
    const double gj = g[j];
    g[j + 1] = -s * gj;
    g[j] = c * gj;
    const double est = fabs(g[j + 1]) / *bnorm;
    stat->iters = j + 1;
    stat->est = est;
    if (!isfinite(est) || !isfinite(hn)) {
      stat->status = WC4D_ERR_NONFINITE;
      stat->done = 1;
    } else if (est <= stat->tol_est || hn == 0.0) {
      stat->done = 1;
    }
  }
  __syncthreads();
  double* out = H + (int64_t)j * ldh;
  for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) out[i] = col[i];
}
void gm_hessenberg(int j, const double* h1, const double* h2, const double* part_norm, double* H, int ldh, double* cs,
                   double* sn, double* g, double* hnext, DevStatus* stat, const double* bnorm, cudaStream_t st) {
  gm_hessenberg_kernel<<<1, DOT_THREADS, sizeof(double) * (3 * (size_t)j + 2), st>>>(j, h1, h2, part_norm, H, ldh,
                                                                                       cs, sn, g, hnext, stat, bnorm);
  WC4D_LAUNCH_CHECK();
}

template <typename T>
__global__ void gm_normalize_kernel(const T* __restrict__ w, const double* hnext, T* __restrict__ v, int64_t n,
                                    const int* done) {
  if (done != nullptr && *(volatile const int*)done) return;
  const double h = *hnext;
  const double ih = h > 0.0 ? 1.0 / h : 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    v[e] = (T)((double)w[e] * ih);
}
template <typename T>
void gm_normalize(const T* w, const double* hnext, T* v, int64_t n, const int* done, cudaStream_t st) {
  const int nb = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  gm_normalize_kernel<T><<<nb, 256, 0, st>>>(w, hnext, v, n, done);
  WC4D_LAUNCH_CHECK();
}
template void gm_normalize<double>(const double*, const double*, double*, int64_t, const int*, cudaStream_t);
template void gm_normalize<float>(const float*, const double*, float*, int64_t, const int*, cudaStream_t);

// y = R^{-1} g[0:k] with R the rotated (upper triangular) k x k Hessenberg
// block: column-oriented back substitution, one block, the right-hand side in
// shared memory.
__global__ void gm_solve_y_kernel(const double* H, int ldh, const double* g, int k, double* y) {
  extern __shared__ double rhs[];
  for (int i = threadIdx.x; i < k; i += blockDim.x) rhs[i] = g[i];
  __syncthreads();
  for (int i = k - 1; i >= 0; --i) {
    const double yi = rhs[i] / H[i + (int64_t)i * ldh];
    __syncthreads();
    for (int r = threadIdx.x; r < i; r += blockDim.x) rhs[r] -= H[r + (int64_t)i * ldh] * yi;
    if (threadIdx.x == 0) y[i] = yi;
    __syncthreads();
  }
}
void gm_solve_y(const double* H, int ldh, const double* g, int k, double* y, cudaStream_t st) {
  gm_solve_y_kernel<<<1, 256, sizeof(double) * (size_t)std::max(k, 1), st>>>(H, ldh, g, k, y);
  WC4D_LAUNCH_CHECK();
}

__global__ void gm_solve_y_dev_kernel(const double* H, int ldh, const double* g, const DevStatus* stat, int kmax,
                                      double* y) {
  extern __shared__ double rhs[];
  const int k = min(stat->iters, kmax);
  for (int i = threadIdx.x; i < k; i += blockDim.x) rhs[i] = g[i];
  __syncthreads();
  for (int i = k - 1; i >= 0; --i) {
    const double yi = rhs[i] / H[i + (int64_t)i * ldh];
    __syncthreads();
    for (int r = threadIdx.x; r < i; r += blockDim.x) rhs[r] -= H[r + (int64_t)i * ldh] * yi;
    if (threadIdx.x == 0) y[i] = yi;
    __syncthreads();
  }
}
void gm_solve_y_dev(const double* H, int ldh, const double* g, const DevStatus* stat, int kmax, double* y,
                    cudaStream_t st) {
  gm_solve_y_dev_kernel<<<1, 256, sizeof(double) * (size_t)std::max(kmax, 1), st>>>(H, ldh, g, stat, kmax, y);
  WC4D_LAUNCH_CHECK();
}

template <typename T, typename TZ>
__global__ void __launch_bounds__(256) gm_combine_dev_kernel(const TZ* __restrict__ Z, int64_t ldz,
                                                             const DevStatus* stat, int kmax,
                                                             const double* __restrict__ y, T* x, int64_t n) {
  extern __shared__ double ys[];
  const int k = min(stat->iters, kmax);
  for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = y[i];
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < k; ++i) acc += ys[i] * (double)Z[(int64_t)i * ldz + e];
    x[e] = (T)acc;
  }
}
template <typename T, typename TZ>
void gm_combine_dev(const TZ* Z, int64_t ldz, const DevStatus* stat, int kmax, const double* y, T* x, int64_t n,
                    cudaStream_t st) {
  const int nb = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  gm_combine_dev_kernel<T, TZ><<<nb, 256, sizeof(double) * std::max(kmax, 1), st>>>(Z, ldz, stat, kmax, y, x, n);
  WC4D_LAUNCH_CHECK();
}
template void gm_combine_dev<double, float>(const float*, int64_t, const DevStatus*, int, const double*, double*,
                                            int64_t, cudaStream_t);

// x = x0 + sum_i y_i Z_i
template <typename T, typename TZ>
__global__ void __launch_bounds__(256) gm_combine_kernel(const TZ* __restrict__ Z, int64_t ldz, int k,
                                                         const double* __restrict__ y, const T* x0, T* x, int64_t n) {
  extern __shared__ double ys[];
  for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = y[i];
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double acc = x0 ? (double)x0[e] : 0.0;
    for (int i = 0; i < k; ++i) acc += ys[i] * (double)Z[(int64_t)i * ldz + e];
    x[e] = (T)acc;
  }
}
template <typename T, typename TZ>
void gm_combine(const TZ* Z, int64_t ldz, int k, const double* y, const T* x0, T* x, int64_t n, cudaStream_t st) {
  const int nb = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  gm_combine_kernel<T, TZ><<<nb, 256, sizeof(double) * std::max(k, 1), st>>>(Z, ldz, k, y, x0, x, n);
  WC4D_LAUNCH_CHECK();
}
template void gm_combine<double, double>(const double*, int64_t, int, const double*, const double*, double*, int64_t,
                                         cudaStream_t);
template void gm_combine<float, float>(const float*, int64_t, int, const double*, const float*, float*, int64_t,
                                       cudaStream_t);
template void gm_combine<double, float>(const float*, int64_t, int, const double*, const double*, double*, int64_t,
                                        cudaStream_t);

// ------------------------------------------------ double-float Arnoldi passes
// The same error-free multiply-add as the double-float GEMM (df_mac /
// df_mac2 in common.cuh): product error by FMA, cross terms, TwoSum into (s, c).
// The same error-free multiply-add as the double-float GEMM: product error by
// FMA, cross terms, Knuth TwoSum into (s, c).


// Block dots V^T w over the split basis.  Grid (chunks of 1024 elements,
// groups of ORTH_G vectors); each thread takes 4 consecutive elements, so every
// basis access is a 16-byte load (the many-stream read pattern reaches HBM
// rate only with wide per-thread loads).  ldv and the buffers are padded to a
// multiple of 4 elements with zeros.
__global__ void __launch_bounds__(DOT_THREADS) gm_mdot_df_kernel(const float* __restrict__ Vh,
                                                                 const float* __restrict__ Vl, int64_t ldv, int cnt,
                                                                 const float* __restrict__ wh,
                                                                 const float* __restrict__ wl, int64_t n4,
                                                                 double* __restrict__ part, const int* done,
                                                                 int* ran) {
  if (done != nullptr && *(volatile const int*)done) return;
  if (ran != nullptr && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *ran = 1;
  __shared__ double sh[DOT_THREADS / 32][ORTH_G];
  const int chunk = blockIdx.x, i0 = blockIdx.y * ORTH_G;
  const int gn = min(ORTH_G, cnt - i0);
  float s[ORTH_G], c[ORTH_G];
#pragma unroll
  for (int g = 0; g < ORTH_G; ++g) s[g] = c[g] = 0.f;
  for (int64_t q = (int64_t)chunk * DOT_THREADS + threadIdx.x; q < n4; q += (int64_t)gridDim.x * DOT_THREADS) {
    const float4 xh = reinterpret_cast<const float4*>(wh)[q];
    const float4 xl = reinterpret_cast<const float4*>(wl)[q];
#pragma unroll
    for (int g = 0; g < ORTH_G; ++g) {
      if (g < gn) {
        const float4 a = reinterpret_cast<const float4*>(Vh + (int64_t)(i0 + g) * ldv)[q];
        const float4 b = reinterpret_cast<const float4*>(Vl + (int64_t)(i0 + g) * ldv)[q];
        df_mac(s[g], c[g], a.x, b.x, xh.x, xl.x);
        df_mac(s[g], c[g], a.y, b.y, xh.y, xl.y);
        df_mac(s[g], c[g], a.z, b.z, xh.z, xl.z);
        df_mac(s[g], c[g], a.w, b.w, xh.w, xl.w);
      }
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int g = 0; g < ORTH_G; ++g) {
    const float2 v = df_warp_sum(s[g], c[g]);
    if (lane == 0) sh[wid][g] = (double)v.x + (double)v.y;
  }
  __syncthreads();
  if (threadIdx.x < ORTH_G && i0 + threadIdx.x < cnt) {
    double v = 0.0;
    for (int k = 0; k < DOT_THREADS / 32; ++k) v += sh[k][threadIdx.x];
    part[(int64_t)(i0 + threadIdx.x) * gridDim.x + chunk] = v;
  }
}
void gm_mdot_df(const float* Vh, const float* Vl, int64_t ldv, int cnt, const float* wh, const float* wl, int64_t n,
                double* part, const int* done, cudaStream_t st) {
  int* ran = prof_begin(PROF_ORTH, (double)(cnt + 1) * n * 8.0, st);
  const int64_t n4 = (n + 3) / 4;
  dim3 grid((unsigned)dot_chunks(n, cnt), (cnt + ORTH_G - 1) / ORTH_G);
  gm_mdot_df_kernel<<<grid, DOT_THREADS, 0, st>>>(Vh, Vl, ldv, cnt, wh, wl, n4, part, done, ran);
  WC4D_LAUNCH_CHECK();
  if (ran) prof_end(st);
}

// w -= V h with double-float accumulation of V h (4 elements per thread,
// 16-byte basis loads), then w is re-split for the next pass
__global__ void __launch_bounds__(DOT_THREADS) gm_mupdate_df_kernel(const float* __restrict__ Vh,
                                                                    const float* __restrict__ Vl, int64_t ldv,
                                                                    int cnt, const double* __restrict__ h,
                                                                    double* __restrict__ w, float* __restrict__ wh,
                                                                    float* __restrict__ wl, int64_t n,
                                                                    const int* done, int* ran) {
  if (done != nullptr && *(volatile const int*)done) return;
  if (ran != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *ran = 1;
  extern __shared__ float hsh[];  // [cnt] hi, [cnt] lo
  float* hsl = hsh + cnt;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    const float hi = __double2float_rn(h[i]);
    hsh[i] = hi;
    hsl[i] = __double2float_rn(h[i] - (double)hi);
  }
  __syncthreads();
  const int64_t n4 = (n + 3) / 4;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n4; q += (int64_t)gridDim.x * blockDim.x) {
    float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
    int i = 0;
    // eight basis vectors per step: sixteen 16-byte loads in flight per thread
    for (; i + 8 <= cnt; i += 8) {
      float4 a[8], b[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        a[u] = reinterpret_cast<const float4*>(Vh + (int64_t)(i + u) * ldv)[q];
        b[u] = reinterpret_cast<const float4*>(Vl + (int64_t)(i + u) * ldv)[q];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float hh = hsh[i + u], hl = hsl[i + u];
        df_mac(s[0], c[0], hh, hl, a[u].x, b[u].x);
        df_mac(s[1], c[1], hh, hl, a[u].y, b[u].y);
        df_mac(s[2], c[2], hh, hl, a[u].z, b[u].z);
        df_mac(s[3], c[3], hh, hl, a[u].w, b[u].w);
      }
    }
    for (; i < cnt; ++i) {
      const float4 a = reinterpret_cast<const float4*>(Vh + (int64_t)i * ldv)[q];
      const float4 b = reinterpret_cast<const float4*>(Vl + (int64_t)i * ldv)[q];
      const float hh = hsh[i], hl = hsl[i];
      df_mac(s[0], c[0], hh, hl, a.x, b.x);
      df_mac(s[1], c[1], hh, hl, a.y, b.y);
      df_mac(s[2], c[2], hh, hl, a.z, b.z);
      df_mac(s[3], c[3], hh, hl, a.w, b.w);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t e = 4 * q + u;
      if (e < n) {
        const double v = w[e] - ((double)s[u] + (double)c[u]);
        w[e] = v;
        const float vh = __double2float_rn(v);
        wh[e] = vh;
        wl[e] = __double2float_rn(v - (double)vh);
      }
    }
  }
}
void gm_mupdate_df(const float* Vh, const float* Vl, int64_t ldv, int cnt, const double* h, double* w, float* wh,
                   float* wl, int64_t n, const int* done, cudaStream_t st) {
  int* ran = prof_begin(PROF_ORTH, (double)cnt * n * 8.0 + 3.0 * n * 8.0, st);
  const int64_t n4 = (n + 3) / 4;
  const int nb = (int)std::min<int64_t>((n4 + DOT_THREADS - 1) / DOT_THREADS, 152 * 16);
  gm_mupdate_df_kernel<<<nb, DOT_THREADS, sizeof(float) * 2 * std::max(cnt, 1), st>>>(Vh, Vl, ldv, cnt, h, w, wh, wl,
                                                                                    n, done, ran);
  WC4D_LAUNCH_CHECK();
  if (ran) prof_end(st);
}

__global__ void gm_normalize_df_kernel(const double* __restrict__ w, const double* hnext, double* __restrict__ v,
                                       float* __restrict__ vh, float* __restrict__ vl, int64_t n, const int* done) {
  if (done != nullptr && *(volatile const int*)done) return;
  const double hh = *hnext;
  const double ih = hh > 0.0 ? 1.0 / hh : 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double x = w[e] * ih;
    v[e] = x;
    const float xh = __double2float_rn(x);
    vh[e] = xh;
    vl[e] = __double2float_rn(x - (double)xh);
  }
}
void gm_normalize_df(const double* w, const double* hnext, double* v, float* vh, float* vl, int64_t n,
                     const int* done, cudaStream_t st) {
  const int nb = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  gm_normalize_df_kernel<<<nb, 256, 0, st>>>(w, hnext, v, vh, vl, n, done);
  WC4D_LAUNCH_CHECK();
}

__global__ void gm_split_kernel(const double* __restrict__ w, float* __restrict__ wh, float* __restrict__ wl, int64_t n,
                                const int* done) {
  if (done != nullptr && *(volatile const int*)done) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double x = w[e];
    const float xh = __double2float_rn(x);
    wh[e] = xh;
    wl[e] = __double2float_rn(x - (double)xh);
  }
}
// the first basis vector with BF16 low parts (the 6-byte basis)
__global__ void gm_split_b6_kernel(const double* __restrict__ w, float* __restrict__ wh, uint16_t* __restrict__ wl,
                                   int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double x = w[e];
    const float xh = __double2float_rn(x);
    wh[e] = xh;
    wl[e] = __bfloat16_as_ushort(__float2bfloat16_rn(__double2float_rn(x - (double)xh)));
  }
}
void gm_split_basis(const double* w, float* vh, float* vl, int64_t n, bool b6, cudaStream_t st) {
  if (!b6) {
    gm_split(w, vh, vl, n, nullptr, st);
    return;
  }
  const int nb = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  gm_split_b6_kernel<<<nb, 256, 0, st>>>(w, vh, reinterpret_cast<uint16_t*>(vl), n);
  WC4D_LAUNCH_CHECK();
}
void gm_split(const double* w, float* wh, float* wl, int64_t n, const int* done, cudaStream_t st) {
  const int nb = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  gm_split_kernel<<<nb, 256, 0, st>>>(w, wh, wl, n, done);
  WC4D_LAUNCH_CHECK();
}

// ------------------------------------------- delayed CGS2 Arnoldi (DF32 GMRES)
// Classical Gram-Schmidt with the reorthogonalisation of each basis vector
// delayed by one step (low-synchronisation CGS2, Bielich, Langou, Thomas,
// Swirydowicz, Yamazaki and Boman, Parallel Computing 2022).  Step j applies the
// operator to the candidate u_j (one projection done, not yet reorthogonalised)
// and reads the basis twice instead of four times:
//   dot pass:    a = [Q_j u_j]^T w,  c = [Q_j u_j]^T u_j,  w^T w
//   coefficients: gamma = |u_j - Q_j c| (Pythagoras), q_j = (u_j - Q_j c)/gamma,
//                b = Q_{j+1}^T w, Hessenberg column j-1 completed (see below)
//   update pass: q_j and the next candidate u_{j+1} = (w - Q_{j+1} b) / alpha
// The operator was applied to u_j, not q_j, so column j-1 of the Hessenberg
// matrix is completed one step late from the identity
//   A P^-1 q_{j-1} = Q_j (b_{j-1} - Hbar c_{j-1} + alpha_j c_j) / gamma_{j-1}
//                    + (alpha_j gamma_j / gamma_{j-1}) q_j,
// Hbar being the unrotated Hessenberg columns 0..j-2.  The preconditioned
// candidates Z~_j = P^-1 u_j are stored as computed; with U = Q T (T upper
// triangular, columns [c_j; gamma_j]) the solution is x0 + Z~ T^-1 y, so the
// rounding of the preconditioner never enters the residual (as in CGS2 GMRES,
// where Z holds the computed P^-1 q_j).

// Low parts of the split basis, four entries at a time: FP32 (8-byte basis
// entries) or, with B6, BF16 (6-byte entries: the low-part array holds 16-bit
// words with the same leading dimension in elements, so a column's low parts
// take half the bytes).  off: first element of the column.
template <bool B6>
__device__ __forceinline__ float4 lo_load(const float* Vl, int64_t off, int64_t q) {
  if constexpr (B6) {
    const uint2 r = reinterpret_cast<const uint2*>(reinterpret_cast<const uint16_t*>(Vl) + off)[q];
    return make_float4(__uint_as_float(r.x << 16), __uint_as_float(r.x & 0xFFFF0000u), __uint_as_float(r.y << 16),
                       __uint_as_float(r.y & 0xFFFF0000u));
  } else {
    return reinterpret_cast<const float4*>(Vl + off)[q];
  }
}
template <bool B6>
__device__ __forceinline__ void lo_store(float* Vl, int64_t off, int64_t q, float4 v) {
  if constexpr (B6) {
    const uint32_t a = __bfloat16_as_ushort(__float2bfloat16_rn(v.x)), b = __bfloat16_as_ushort(__float2bfloat16_rn(v.y));
    const uint32_t c = __bfloat16_as_ushort(__float2bfloat16_rn(v.z)), d = __bfloat16_as_ushort(__float2bfloat16_rn(v.w));
    reinterpret_cast<uint2*>(reinterpret_cast<uint16_t*>(Vl) + off)[q] = make_uint2(a | (b << 16), c | (d << 16));
  } else {
    reinterpret_cast<float4*>(Vl + off)[q] = v;
  }
}

// asynchronous global -> shared copies of 16 and 8 bytes (cp.async; the
// issuing thread waits for its own groups with cp.async.wait_group)
__device__ __forceinline__ void cpa16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cpa8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
constexpr int DC_NS = 2;                    // stages of each thread's private copy ring
constexpr int DC_SLOTS = 2 * ORTH_G + 4;    // per stage: G basis hi, G basis lo, w hi, w lo, u hi, u lo
constexpr size_t DC_DOT_SMEM = (size_t)DC_NS * DC_SLOTS * DOT_THREADS * 16;
// part rows: a_0..a_j | c_0..c_j (c_j = u_j^T u_j) | w^T w.  The pass is
// bound by the bytes in flight per SM: each thread keeps its next stage of
// entries in flight through a private shared-memory ring (two stages, 96 KB
// per CTA, two CTAs per SM) instead of in registers (39.1 against 44.3 us per
// pass at the scale window, the update pass unchanged).
template <bool B6>
__global__ void __launch_bounds__(DOT_THREADS, 2) gm_dc_dot_kernel(const float* __restrict__ Vh,
                                                                const float* __restrict__ Vl, int64_t ldv, int j,
                                                                const float* __restrict__ wh,
                                                                const float* __restrict__ wl, int64_t n4,
                                                                float2* __restrict__ part, const int* done,
                                                                int* ran) {
  pdl_wait();
  pdl_trigger();
  if (done != nullptr && *(volatile const int*)done) return;
  if (ran != nullptr && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *ran = 1;
  __shared__ float2 sh[DOT_THREADS / 32][2 * ORTH_G + 1];
  const int cnt = j + 1;
  const int chunk = blockIdx.x, i0 = blockIdx.y * ORTH_G;
  const int gn = min(ORTH_G, cnt - i0);
  const bool first = blockIdx.y == 0;
  // double-float accumulators: per basis vector one paired (against w, against
  // u) accumulator, so one paired multiply-add (FFMA2 / FADD2: each lane rounds
  // as its scalar form) serves both dot products of a basis entry, at the
  // register count of the scalar form; w^T w in a scalar pair
  float2 s2[ORTH_G], c2[ORTH_G];
  float s[2 * ORTH_G + 1], c[2 * ORTH_G + 1];
#pragma unroll
  for (int g = 0; g < ORTH_G; ++g) s2[g] = c2[g] = make_float2(0.f, 0.f);
  s[2 * ORTH_G] = c[2 * ORTH_G] = 0.f;
  const float* uhp = Vh + (int64_t)j * ldv;
  // every thread streams its own entries through a private ring of DC_NS
  // stages in shared memory with asynchronous 16-byte copies (8-byte for BF16
  // low parts): the loads of the next stages are in flight while this one is
  // summed, and no register holds a load in flight
  extern __shared__ float4 dring[];  // [DC_NS][DC_SLOTS][DOT_THREADS]
  const int tid = threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * DOT_THREADS;
  const int64_t qbeg = (int64_t)chunk * DOT_THREADS + tid;
  auto issue = [&](int stg, int64_t q) {
    if (q < n4) {
      float4* S = dring + (size_t)stg * DC_SLOTS * DOT_THREADS + tid;
#pragma unroll
      for (int g = 0; g < ORTH_G; ++g) {
        if (g < gn) {
          cpa16(S + g * DOT_THREADS, Vh + (int64_t)(i0 + g) * ldv + 4 * q);
          if constexpr (B6)
            cpa8(S + (ORTH_G + g) * DOT_THREADS, reinterpret_cast<const uint16_t*>(Vl) + (int64_t)(i0 + g) * ldv + 4 * q);
          else
            cpa16(S + (ORTH_G + g) * DOT_THREADS, Vl + (int64_t)(i0 + g) * ldv + 4 * q);
        }
      }
      cpa16(S + (2 * ORTH_G) * DOT_THREADS, wh + 4 * q);
      cpa16(S + (2 * ORTH_G + 1) * DOT_THREADS, wl + 4 * q);
      cpa16(S + (2 * ORTH_G + 2) * DOT_THREADS, uhp + 4 * q);
      if constexpr (B6)
        cpa8(S + (2 * ORTH_G + 3) * DOT_THREADS, reinterpret_cast<const uint16_t*>(Vl) + (int64_t)j * ldv + 4 * q);
      else
        cpa16(S + (2 * ORTH_G + 3) * DOT_THREADS, Vl + (int64_t)j * ldv + 4 * q);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  auto lo_of = [&](const float4* p) -> float4 {
    if constexpr (B6) {
      const uint2 r = *reinterpret_cast<const uint2*>(p);
      return make_float4(__uint_as_float(r.x << 16), __uint_as_float(r.x & 0xFFFF0000u), __uint_as_float(r.y << 16),
                         __uint_as_float(r.y & 0xFFFF0000u));
    } else {
      return *p;
    }
  };
#pragma unroll
  for (int st0 = 0; st0 < DC_NS - 1; ++st0) issue(st0, qbeg + st0 * stride);
  int stg = 0;
  for (int64_t q = qbeg; q < n4; q += stride) {
    issue((stg + DC_NS - 1) % DC_NS, q + (DC_NS - 1) * stride);
    asm volatile("cp.async.wait_group %0;" ::"n"(DC_NS - 1) : "memory");
    const float4* S = dring + (size_t)stg * DC_SLOTS * DOT_THREADS + tid;
    stg = (stg + 1) % DC_NS;
    const float4 xh = S[(2 * ORTH_G) * DOT_THREADS];
    const float4 xl = S[(2 * ORTH_G + 1) * DOT_THREADS];
    const float4 uh = S[(2 * ORTH_G + 2) * DOT_THREADS];
    const float4 ul = lo_of(S + (2 * ORTH_G + 3) * DOT_THREADS);
#pragma unroll
    for (int g = 0; g < ORTH_G; ++g) {
      if (g < gn) {
        const float4 a = S[g * DOT_THREADS];
        const float4 b = lo_of(S + (ORTH_G + g) * DOT_THREADS);
        df_mac2(s2[g], c2[g], make_float2(a.x, a.x), make_float2(b.x, b.x), make_float2(xh.x, uh.x),
                make_float2(xl.x, ul.x));
        df_mac2(s2[g], c2[g], make_float2(a.y, a.y), make_float2(b.y, b.y), make_float2(xh.y, uh.y),
                make_float2(xl.y, ul.y));
        df_mac2(s2[g], c2[g], make_float2(a.z, a.z), make_float2(b.z, b.z), make_float2(xh.z, uh.z),
                make_float2(xl.z, ul.z));
        df_mac2(s2[g], c2[g], make_float2(a.w, a.w), make_float2(b.w, b.w), make_float2(xh.w, uh.w),
                make_float2(xl.w, ul.w));
      }
    }
    if (first) {
      df_mac(s[2 * ORTH_G], c[2 * ORTH_G], xh.x, xl.x, xh.x, xl.x);
      df_mac(s[2 * ORTH_G], c[2 * ORTH_G], xh.y, xl.y, xh.y, xl.y);
      df_mac(s[2 * ORTH_G], c[2 * ORTH_G], xh.z, xl.z, xh.z, xl.z);
      df_mac(s[2 * ORTH_G], c[2 * ORTH_G], xh.w, xl.w, xh.w, xl.w);
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");  // no copy in flight past the loop
  // warp reduction in double-float on the FP32 pipe (an FP64 shuffle tree per
  // vector would occupy GB300's 1/64-rate FP64 pipe for a large part of the
  // kernel); one FP64 conversion per warp and vector
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int g = 0; g < ORTH_G; ++g) {
    s[g] = s2[g].x;
    c[g] = c2[g].x;
    s[ORTH_G + g] = s2[g].y;
    c[ORTH_G + g] = c2[g].y;
  }
#pragma unroll
  for (int g = 0; g < 2 * ORTH_G + 1; ++g) {
    const float2 v = df_warp_sum(s[g], c[g]);
    if (lane == 0) sh[wid][g] = v;
  }
  __syncthreads();
  const int r = threadIdx.x;  // threads 0..2*ORTH_G of warp 0: one FP64 conversion each
  if (r < 2 * ORTH_G + 1) {
    float2 a2 = sh[0][r];
    for (int k = 1; k < DOT_THREADS / 32; ++k) a2 = df_add(a2, sh[k][r]);
    int row = -1;
    if (r < ORTH_G) {
      if (r < gn) row = i0 + r;
    } else if (r < 2 * ORTH_G) {
      if (r - ORTH_G < gn) row = cnt + i0 + r - ORTH_G;
    } else if (first) {
      row = 2 * cnt;
    }
    if (row >= 0) part[(int64_t)row * gridDim.x + chunk] = a2;  // summed by the coefficient kernel
  }
}
void gm_dc_dot(const float* Vh, const float* Vl, int64_t ldv, int j, const float* wh, const float* wl, int64_t n,
               float2* part, const int* done, cudaStream_t st, bool b6) {
  // profiled bytes: the FP64-equivalent 8 B per basis entry in both forms
  int* ran = prof_begin(PROF_ORTH, (double)(j + 3) * n * 8.0, st, b6 ? (double)(j + 2) * n * 6.0 + (double)n * 8.0 : 0.0);
  const int64_t n4 = (n + 3) / 4;
  dim3 grid((unsigned)dc_dot_chunks(n, j + 1), (j + 1 + ORTH_G - 1) / ORTH_G);
  static std::once_flag once;
  std::call_once(once, [] {
    WC4D_CUDA(cudaFuncSetAttribute(gm_dc_dot_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DC_DOT_SMEM));
    WC4D_CUDA(cudaFuncSetAttribute(gm_dc_dot_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DC_DOT_SMEM));
  });
  if (b6)
    WC4D_CUDA(launch_pdl(gm_dc_dot_kernel<true>, grid, dim3(DOT_THREADS), DC_DOT_SMEM, st, Vh, Vl, ldv, j, wh, wl, n4, part,
                         done, ran));
  else
    WC4D_CUDA(launch_pdl(gm_dc_dot_kernel<false>, grid, dim3(DOT_THREADS), DC_DOT_SMEM, st, Vh, Vl, ldv, j, wh, wl, n4,
                         part, done, ran));
  WC4D_LAUNCH_CHECK();
  if (ran) prof_end(st);
}

// Applies the Givens rotations 0..m-1 (cosines rc, sines rs) to a new
// Hessenberg column col[0..m] in place.  Rotation i maps the pair
// (a_i, col[i+1]) to (rc_i a_i + rs_i col[i+1], -rs_i a_i + rc_i col[i+1]),
// where a_0 = col[0] and a_{i+1} is the second component: an affine recurrence
// a_{i+1} = alpha_i a_i + beta_i with alpha_i = -rs_i, beta_i = rc_i col[i+1].
// Affine maps compose associatively, so the chain is an inclusive scan of
// (A, B) pairs (a -> A a + B) instead of m dependent steps: on GB300 a serial
// FP64 chain in one thread costs tens of cycles per operation.  Only the
// first nt threads (a multiple of 32, as few as keep at most SCAN_PER
// rotations per thread) take part: GB300 issues one warp FP64 instruction
// per 16 SM cycles, so every idle warp's share of the scan would be pure
// cost.  Every thread of the block must call it (it has block barriers).
// Ends with col[0..m-1] rotated and col[m] = a_m; col[m+1] is untouched.
// Needs m <= SCAN_PER * blockDim.x; sh: 64 doubles of shared scratch.
constexpr int SCAN_PER = 8;
__device__ void rotate_column_scan(double* col, const double* rc, const double* rs, int m, double* sh) {
  const int nt = min((int)blockDim.x, 32 * ((m + 32 * SCAN_PER - 1) / (32 * SCAN_PER)));
  const int per = (m + nt - 1) / nt;  // at most SCAN_PER rotations per thread
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwa = nt >> 5;
  const bool act = (int)threadIdx.x < nt;  // warp-uniform
  const int i0 = threadIdx.x * per;
  const int i1 = act ? min(i0 + per, m) : i0;
  double A = 1.0, B = 0.0;
  double* wa = sh;
  double* wb = sh + 32;
  if (act) {
    for (int i = i0; i < i1; ++i) {  // this thread's rotations composed, in order
      const double al = -rs[i], be = rc[i] * col[i + 1];
      B = al * B + be;
      A = al * A;
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {  // inclusive scan within the warp: later o earlier
      const double Ap = __shfl_up_sync(0xffffffffu, A, off), Bp = __shfl_up_sync(0xffffffffu, B, off);
      if (lane >= off) {
        B = A * Bp + B;
        A = A * Ap;
      }
    }
  }
  __syncthreads();  // sh may hold a previous reduction's partials
  if (act && lane == 31) {
    wa[wid] = A;
    wb[wid] = B;
  }
  __syncthreads();
  if (wid == 0 && nwa > 1) {
    double X = lane < nwa ? wa[lane] : 1.0, Y = lane < nwa ? wb[lane] : 0.0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const double Xp = __shfl_up_sync(0xffffffffu, X, off), Yp = __shfl_up_sync(0xffffffffu, Y, off);
      if (lane >= off) {
        Y = X * Yp + Y;
        X = X * Xp;
      }
    }
    if (lane < nwa) {
      wa[lane] = X;
      wb[lane] = Y;
    }
  }
  __syncthreads();
  double outv[SCAN_PER];
  double av = 0.0;
  if (act) {
    // exclusive prefix of this thread = (lane-exclusive within the warp) o (warps before)
    double eA = __shfl_up_sync(0xffffffffu, A, 1), eB = __shfl_up_sync(0xffffffffu, B, 1);
    if (lane == 0) {
      eA = 1.0;
      eB = 0.0;
    }
    if (wid > 0) {
      const double PA = wa[wid - 1], PB = wb[wid - 1];
      eB = eA * PB + eB;
      eA = eA * PA;
    }
    av = eA * col[0] + eB;  // a_{i0}
    for (int i = i0; i < i1; ++i) {
      const double y = col[i + 1];
      outv[i - i0] = rc[i] * av + rs[i] * y;
      av = -rs[i] * av + rc[i] * y;
    }
  }
  __syncthreads();  // every thread has read the unrotated column
  for (int i = i0; i < i1; ++i) col[i] = outv[i - i0];
  if (act && i0 < m && i1 == m) col[m] = av;
  __syncthreads();
}

// One CTA.  part: the dot pass's per-chunk partials (double-float pairs,
// nchunks per row; rows a_0..a_j | c_0..c_j | w^T w).  dc: scalar state
// (DC_* slots), bprev / cprev: b and c of the previous step, e: the update
// coefficients.  Sums the partials (the dot reduction), completes Hessenberg
// column j-1 (raw into Hraw, rotated into H), updates the Givens rotations, g
// and the status, and writes column j of the triangular T with
// u_j = Q_j c_j + gamma_j q_j (T = [c_j; gamma_j]), so that P^-1 Q = Z~ T^-1
// for the stored Z~_j = P^-1 u_j.  GB300 issues one warp FP64 instruction per
// 16 SM cycles, so the FP64 work is laid out by instruction count: the sums
// of the partials run in double-float on the FP32 pipe (one FP64 conversion
// per row), the scalar chain runs in one warp, not redundantly in eight.
// Shared memory: the reduced rows, the column, the rotations, b and Hbar c
// of the previous step (7 j + 5 doubles), then the staged partials.
__global__ void __launch_bounds__(256) gm_dc_coef_kernel(int j, const float2* __restrict__ part, int nchunks,
                                                         double* dc, double* bprev, double* cprev, double* e,
                                                         double* Hraw, double* H, double* T, int ldh, double* cs,
                                                         double* sn, double* g, double* hnext, DevStatus* stat,
                                                         const double* bnorm, const double* __restrict__ hc) {
  extern __shared__ double sm[];
  __shared__ double sh[64];
  __shared__ double scal[4];
  __shared__ double pre[8];  // dc[ALPHA], dc[GAMMA], dc[BETA], g[j-1], ||b||, tol_est
  __shared__ int sdone;
  pdl_wait();
  pdl_trigger();
  const int cnt = j + 1, rows = 2 * cnt + 1;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double* red = sm;           // [2 j + 3]: a_0..a_j | c_0..c_j | w^T w
  double* col = red + rows;   // [j + 2]
  double* rc = col + j + 2;   // [j]
  double* rs = rc + j;        // [j]
  double* bp = rs + j;        // [j]: b of the previous step
  double* hcs = bp + j;       // [j]: Hbar c of the previous step
  // every operand the kernel reads, in flight at once: the serial chain
  // below then waits on shared memory, not on a global round trip per use
  if (threadIdx.x == 0) {
    sdone = *(volatile const int*)&stat->done;
    pre[0] = dc[DC_ALPHA];
    pre[1] = dc[DC_GAMMA];
    pre[2] = dc[DC_BETA];
    pre[3] = j >= 1 ? g[j - 1] : 0.0;
    pre[4] = *bnorm;
    pre[5] = stat->tol_est;
  }
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    if (i + 1 < j) {
      rc[i] = cs[i];
      rs[i] = sn[i];
    }
    bp[i] = bprev[i];
    hcs[i] = j >= 2 ? hc[i] : 0.0;
  }
  // the dot reduction: the whole partial block (rows x nchunks pairs, at most
  // about 5.5k) is staged in shared memory by every thread with eight loads
  // in flight each, then each row is summed by tpr lanes (a power of two, as
  // many as keep every thread busy) over the chunks in a fixed order
  float2* pst = reinterpret_cast<float2*>(hcs + j);  // [rows * nchunks]
  const int total = rows * nchunks;
  for (int i0 = threadIdx.x; i0 < total; i0 += 8 * blockDim.x) {
    float2 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = i0 + u * blockDim.x;
      v[u] = i < total ? part[i] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i < total) pst[i] = v[u];
    }
  }
  __syncthreads();
  int tpr = 32;
  while (tpr > 1 && tpr * rows > (int)blockDim.x) tpr >>= 1;
  const int sub = lane & (tpr - 1), per_round = blockDim.x / tpr;
  for (int r0 = 0; r0 < rows; r0 += per_round) {
    const int r = r0 + (int)threadIdx.x / tpr;
    float2 acc = make_float2(0.f, 0.f);
    if (r < rows)
      for (int k = sub; k < nchunks; k += tpr) acc = df_add(acc, pst[r * nchunks + k]);
    // rows never straddle a warp (tpr divides 32); lanes past the last row add zeros
    for (int o = tpr >> 1; o > 0; o >>= 1)
      acc = df_add(acc, make_float2(__shfl_xor_sync(0xffffffffu, acc.x, o), __shfl_xor_sync(0xffffffffu, acc.y, o)));
    if (sub == 0 && r < rows) red[r] = (double)acc.x + (double)acc.y;
  }
  __syncthreads();
  if (sdone) return;  // block-uniform
  const double* a = red;        // a_0..a_j
  const double* c = red + cnt;  // c_0..c_{j-1}, c_j = u_j^T u_j
  const double ww = red[2 * cnt];
  const double alpha = pre[0];  // scale of u_j
  const double gprev = pre[1];
  // Independent FP64 chains run in different warps, so their latencies
  // overlap: warp 0 gamma and b_j (and column j-1 from them), warp 1 the
  // reciprocals 1 / gamma_{j-1} and 1 / ||b|| (before warp 0 needs the first),
  // warp 2 the next candidate's scale alpha (after the first barrier).
  if (wid == 1 && lane == 0) {
    pre[6] = 1.0 / gprev;
    pre[7] = 1.0 / pre[4];
  }
  if (wid == 0) {
    // gamma by Pythagoras, b_j = q_j^T w, |b|^2 (one warp; every lane holds the values)
    double cc = 0.0, ca = 0.0, bb = 0.0;
    for (int i = lane; i < j; i += 32) {
      cc += c[i] * c[i];
      ca += c[i] * a[i];
      bb += a[i] * a[i];
    }
    cc = warp_sum(cc);
    ca = warp_sum(ca);
    bb = warp_sum(bb);
    const double g2 = c[j] - cc;
    const double rg = g2 > 0.0 ? rsqrt(g2) : 0.0;  // 1 / gamma
    const double gam = g2 > 0.0 ? g2 * rg : sqrt_clamped(g2);
    const double bj = (a[j] - ca) * rg;
    if (lane == 0) {
      scal[0] = gam;
      scal[1] = rg;
      scal[2] = bj;
      scal[3] = bb + bj * bj;  // |w - Q b|^2 = w^T w - b^T b
    }
  }
  __syncthreads();
  const double gam = scal[0], igam = scal[1], bj = scal[2];
  if (wid == 2 && lane == 0) {
    const double a2 = fmax(ww - scal[3], ww * 1e-30);
    const double ra = a2 > 0.0 ? rsqrt(a2) : 0.0;
    dc[DC_ALPHA] = a2 > 0.0 ? a2 * ra : 1.0;
    dc[DC_IALPHA] = ra;
    dc[DC_GAMMA] = gam;
    dc[DC_IGAMMA] = igam;
  }
  // column j-1: (b_{j-1} - Hbar c_{j-1} + alpha c_j) / gamma_{j-1}, sub-diagonal alpha gamma / gamma_{j-1};
  // hc = Hbar c_{j-1} was formed by the previous step's update kernel (Hbar_{j-1} has no columns at j = 1)
  if (j >= 1) {
    const double ig = pre[6];
    double* raw = Hraw + (int64_t)(j - 1) * ldh;
    for (int r = threadIdx.x; r < j; r += blockDim.x) {
      const double v = (bp[r] - hcs[r] + alpha * c[r]) * ig;
      col[r] = v;
      raw[r] = v;
    }
    if (threadIdx.x == 0) {
      col[j] = alpha * gam * ig;
      raw[j] = col[j];
    }
  }
  {
    double* tc = T + (int64_t)j * ldh;
    for (int r = threadIdx.x; r < j; r += blockDim.x) tc[r] = c[r];
    if (threadIdx.x == 0) tc[j] = gam;
  }
  __syncthreads();
  if (j >= 2) rotate_column_scan(col, rc, rs, j - 1, sh);  // ends with a barrier
  if (threadIdx.x == 0) {
    if (j == 0) {
      g[0] = pre[2] * gam;  // r0 = ||r0|| u_0 = (||r0|| gamma_0) q_0
      stat->iters = 0;
      if (!isfinite(gam) || !isfinite(ww) || !isfinite(bj)) {
        stat->status = WC4D_ERR_NONFINITE;
        stat->done = 1;
      } else if (!(gam > 0.0)) {
        stat->status = WC4D_ERR_BREAKDOWN;
        stat->done = 1;
      }
    } else {
      const int jc = j - 1;  // column being completed (rows 0..jc already rotated)
      *hnext = col[j];
      double cr = 1.0, sr = 0.0;
      const double x = col[jc], y = col[jc + 1];
      if (y != 0.0) {
        // the rotation from 1 / sqrt(x^2 + y^2) (one reciprocal square root instead of hypot and a
        // division); hypot's scaling only where the sum of squares leaves the normal range
        const double s2 = x * x + y * y;
        const double ir = (s2 > 1e-300 && s2 < 1e300) ? rsqrt(s2) : 1.0 / hypot(x, y);
        cr = x * ir;
        sr = y * ir;
      }
      cs[jc] = cr;
      sn[jc] = sr;
      col[jc] = cr * x + sr * y;
      col[jc + 1] = 0.0;
      const double gj = pre[3];
      g[jc + 1] = -sr * gj;
      g[jc] = cr * gj;
      const double est = fabs(sr * gj) * pre[7];
      stat->iters = j;
      stat->est = est;
      if (!isfinite(est) || !isfinite(gam) || !isfinite(ww) || !isfinite(bj)) {
        stat->status = WC4D_ERR_NONFINITE;
        stat->done = 1;
      } else if (est <= pre[5] || !(gam > 0.0)) {
        stat->done = 1;
      }
    }
  }
  // b = (a_0..a_{j-1}, bj) and the update coefficients e' = b - (b_j / gamma) c
  const double ratio = bj * igam;
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    bprev[i] = a[i];
    cprev[i] = c[i];
    e[i] = a[i] - ratio * c[i];
  }
  if (threadIdx.x == 0) {
    bprev[j] = bj;
    e[j] = ratio;
  }
  __syncthreads();
  if (j >= 1) {
    double* out = H + (int64_t)(j - 1) * ldh;
    for (int r = threadIdx.x; r <= j; r += blockDim.x) out[r] = col[r];
  }
}
// (7 j + 5) doubles and (2 j + 3) x nchunks partials (at most about 5.5k: the dot pass's chunk count falls as
// its vector groups grow) for j <= 2000 (GMRES maxit <= 2000)
constexpr int COEF_SMEM_MAX = 160 * 1024;
void gm_dc_coef(int j, const float2* part, int nchunks, double* dc, double* bprev, double* cprev, double* e,
                double* Hraw, double* H, double* T, int ldh, double* cs, double* sn, double* g, double* hnext,
                DevStatus* stat, const double* bnorm, const double* hc, cudaStream_t st) {
  static std::once_flag once;
  std::call_once(once, [] {
    WC4D_CUDA(cudaFuncSetAttribute(gm_dc_coef_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, COEF_SMEM_MAX));
  });
  const size_t smem = sizeof(double) * (7 * (size_t)j + 5) + sizeof(float2) * (2 * (size_t)j + 3) * nchunks;
  WC4D_CHECK(smem <= (size_t)COEF_SMEM_MAX, WC4D_ERR_ARG, "internal: Arnoldi step beyond the coefficient kernel");
  WC4D_CUDA(launch_pdl(gm_dc_coef_kernel, dim3(1), dim3(256), smem, st, j, part, nchunks, dc, bprev, cprev, e, Hraw,
                       H, T, ldh, cs, sn, g, hnext, stat, bnorm, hc));
  WC4D_LAUNCH_CHECK();
}

// q_j = (u_j - Q_j c) / gamma into slot j (in place), u_{j+1} = (w - Q_j e' - e_j u_j) / alpha
// into slot j+1 and into v (double, the next operator input).  Both sums and
// the q_j epilogue in double-float; 2 elements per thread (8-byte loads):
// one float4 per thread gave n/4 threads, about 17 warps per SM at the scale
// window; with a float2 the resident wave of 64-thread CTAs keeps 32 warps'
// loads in flight (orth passes 39.1 -> 38.0 µs mean)
constexpr int UPD_THREADS = 64;
// sixteen 64-thread CTAs per SM (64 registers): 32 warps' loads in flight
template <bool B6>
__global__ void __launch_bounds__(UPD_THREADS, 16) gm_dc_update_kernel(float* Vh, float* Vl, int64_t ldv, int j,
                                                                   const double* __restrict__ e,
                                                                   const double* __restrict__ cv,
                                                                   const double* __restrict__ dc,
                                                                   const double* __restrict__ w,
                                                                   double* __restrict__ v, int64_t n,
                                                                   const double* __restrict__ Hraw, int ldh,
                                                                   double* __restrict__ hc, const int* done,
                                                                   int* ran) {
  pdl_wait();
  pdl_trigger();
  if (done != nullptr && *(volatile const int*)done) return;
  if (ran != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *ran = 1;
  // hc = Hbar_j c_j for the next step's coefficient kernel: raw Hessenberg
  // columns 0..j-1 (rows 0..j) times c_j, one row per block, spread over the grid
  for (int r = blockIdx.x; r <= j && j >= 1; r += gridDim.x) {
    __shared__ double shr[32];
    double t = 0.0;
    for (int k = (r > 0 ? r - 1 : 0) + threadIdx.x; k < j; k += blockDim.x) t += Hraw[r + (int64_t)k * ldh] * cv[k];
    t = block_sum(t, shr);
    if (threadIdx.x == 0) hc[r] = t;
  }
  extern __shared__ float cf[];  // e hi/lo [j], c hi/lo [j]
  float* eh = cf;
  float* el = eh + j;
  float* ch = el + j;
  float* cl = ch + j;
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    const float x = __double2float_rn(e[i]);
    eh[i] = x;
    el[i] = __double2float_rn(e[i] - (double)x);
    const float y = __double2float_rn(cv[i]);
    ch[i] = y;
    cl[i] = __double2float_rn(cv[i] - (double)y);
  }
  __syncthreads();
  // scalars as double-float pairs: the per-element epilogue stays on the FP32 pipe
  const float2 eJ = df_from(e[j]), gI = df_from(dc[DC_IGAMMA]);
  const double ialpha = dc[DC_IALPHA];
  // two elements per thread (one float2 of each basis vector): n/2 threads,
  // about twice the warps per SM of one float4 per thread, for the latency of
  // the basis loads
  const int64_t n2 = (n + 1) / 2;
  float* qh = Vh + (int64_t)j * ldv;
  float* nh = Vh + (int64_t)(j + 1) * ldv;
  auto lo2 = [&](int64_t off, int64_t q) -> float2 {
    if constexpr (B6) {
      const uint32_t r = reinterpret_cast<const uint32_t*>(reinterpret_cast<const uint16_t*>(Vl) + off)[q];
      return make_float2(__uint_as_float(r << 16), __uint_as_float(r & 0xFFFF0000u));
    } else {
      return reinterpret_cast<const float2*>(Vl + off)[q];
    }
  };
  auto lo2_store = [&](int64_t off, int64_t q, float2 v) {
    if constexpr (B6) {
      const uint32_t a = __bfloat16_as_ushort(__float2bfloat16_rn(v.x)), b = __bfloat16_as_ushort(__float2bfloat16_rn(v.y));
      reinterpret_cast<uint32_t*>(reinterpret_cast<uint16_t*>(Vl) + off)[q] = a | (b << 16);
    } else {
      reinterpret_cast<float2*>(Vl + off)[q] = v;
    }
  };
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n2; q += (int64_t)gridDim.x * blockDim.x) {
    float2 se = make_float2(0.f, 0.f), ce = se, sc = se, cc = se;  // paired accumulators: elements 0, 1
    int i = 0;
    // groups of UPD_G basis vectors: 2 UPD_G 8-byte loads in flight per thread
    constexpr int UPD_G = 8;
    for (; i + UPD_G <= j; i += UPD_G) {
      float2 a[UPD_G], b[UPD_G];
#pragma unroll
      for (int u = 0; u < UPD_G; ++u) {
        a[u] = reinterpret_cast<const float2*>(Vh + (int64_t)(i + u) * ldv)[q];
        b[u] = lo2((int64_t)(i + u) * ldv, q);
      }
#pragma unroll
      for (int u = 0; u < UPD_G; ++u) {
        const float2 h1 = make_float2(eh[i + u], eh[i + u]), l1 = make_float2(el[i + u], el[i + u]);
        const float2 h2 = make_float2(ch[i + u], ch[i + u]), l2 = make_float2(cl[i + u], cl[i + u]);
        df_mac2(se, ce, h1, l1, a[u], b[u]);
        df_mac2(sc, cc, h2, l2, a[u], b[u]);
      }
    }
    for (; i < j; ++i) {
      const float2 a = reinterpret_cast<const float2*>(Vh + (int64_t)i * ldv)[q];
      const float2 b = lo2((int64_t)i * ldv, q);
      const float2 h1 = make_float2(eh[i], eh[i]), l1 = make_float2(el[i], el[i]);
      const float2 h2 = make_float2(ch[i], ch[i]), l2 = make_float2(cl[i], cl[i]);
      df_mac2(se, ce, h1, l1, a, b);
      df_mac2(sc, cc, h2, l2, a, b);
    }
    const float se_s[2] = {se.x, se.y}, ce_s[2] = {ce.x, ce.y};
    const float sc_s[2] = {sc.x, sc.y}, cc_s[2] = {cc.x, cc.y};
    const float2 uh = reinterpret_cast<const float2*>(qh)[q];
    const float2 ul = lo2((int64_t)j * ldv, q);
    const float uhs[2] = {uh.x, uh.y}, uls[2] = {ul.x, ul.y};
    float oqh[2], oql[2], onh[2], onl[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t el_ = 2 * q + u;
      const float2 uj = make_float2(uhs[u], uls[u]);
      float2 scs, ses;
      two_sum(sc_s[u], cc_s[u], scs.x, scs.y);
      two_sum(se_s[u], ce_s[u], ses.x, ses.y);
      const float2 qd = df_mul(df_add(uj, df_neg(scs)), gI);  // (u_j - Q_j c) / gamma
      float2 nd = make_float2(0.f, 0.f);
      if (el_ < n) {
        // (w - (Q_j e' + e_j u_j)) / alpha: the projection in double-float, the
        // subtraction from w in FP64 (it cancels when w is nearly in span Q, and
        // w's low bits would be lost in a double-float copy of w)
        const float2 pr = df_add(ses, df_mul(eJ, uj));
        const double nv = (w[el_] - ((double)pr.x + (double)pr.y)) * ialpha;
        v[el_] = nv;
        nd = df_from(nv);
      }
      oqh[u] = qd.x;
      oql[u] = qd.y;
      onh[u] = nd.x;
      onl[u] = nd.y;
    }
    reinterpret_cast<float2*>(qh)[q] = make_float2(oqh[0], oqh[1]);
    lo2_store((int64_t)j * ldv, q, make_float2(oql[0], oql[1]));
    reinterpret_cast<float2*>(nh)[q] = make_float2(onh[0], onh[1]);
    lo2_store((int64_t)(j + 1) * ldv, q, make_float2(onl[0], onl[1]));
  }
}
void gm_dc_update(float* Vh, float* Vl, int64_t ldv, int j, const double* e, const double* c, const double* dc,
                  const double* w, double* v, int64_t n, const double* Hraw, int ldh, double* hc, const int* done,
                  cudaStream_t st, bool b6) {
  // FP64-equivalent bytes: j + 1 basis entries and u_j read, q_j and u_{j+1} written at 8 B, w read, v written;
  // with the 6-byte basis the passes move 6 B per basis entry
  int* ran = prof_begin(PROF_ORTH, (double)(j + 1) * n * 8.0 + 4.0 * n * 8.0, st,
                        b6 ? (double)(j + 1) * n * 6.0 + 2.0 * n * 6.0 + 2.0 * n * 8.0 : 0.0);
  const int64_t n2 = (n + 1) / 2;
  // one resident wave (at most 16 CTAs of 64 threads per SM at 64 registers;
  // fewer once the 16 j bytes of coefficients per CTA limit them), the
  // threads striding over the float2 positions; cached per 4 KB of
  // coefficients (host threads may race to fill an entry, all with one value)
  static std::atomic<int> resident[2][64];
  const int key = (int)std::min<int64_t>(63, (int64_t)16 * j / 4096);
  int res = resident[b6][key].load(std::memory_order_relaxed);
  if (res == 0) {
    int dev = 0, sms = 0, per = 0;
    const size_t smem_key = (size_t)(key + 1) * 4096;  // at least the launch's coefficient bytes
    WC4D_CUDA(cudaGetDevice(&dev));
    WC4D_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (b6)
      WC4D_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, gm_dc_update_kernel<true>, UPD_THREADS, smem_key));
    else
      WC4D_CUDA(
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, gm_dc_update_kernel<false>, UPD_THREADS, smem_key));
    res = std::max(1, sms * std::max(per, 1));
    resident[b6][key].store(res, std::memory_order_relaxed);
  }
  const int nb = (int)std::min<int64_t>((n2 + UPD_THREADS - 1) / UPD_THREADS, res);
  const size_t smem = sizeof(float) * 4 * std::max(j, 1);
  if (b6)
    WC4D_CUDA(launch_pdl(gm_dc_update_kernel<true>, dim3(nb), dim3(UPD_THREADS), smem, st, Vh, Vl, ldv, j, e, c, dc,
                         w, v, n, Hraw, ldh, hc, done, ran));
  else
    WC4D_CUDA(launch_pdl(gm_dc_update_kernel<false>, dim3(nb), dim3(UPD_THREADS), smem, st, Vh, Vl, ldv, j, e, c, dc,
                         w, v, n, Hraw, ldh, hc, done, ran));
  WC4D_LAUNCH_CHECK();
  if (ran) prof_end(st);
}

// ---------------------------------------------------------------- vectors
template <typename T>
__global__ void axpby_kernel(T* y, const T* x, double a, double b, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = (T)(a * (double)x[e] + b * (double)y[e]);
}
template <typename T>
void vec_axpby(T* y, const T* x, double a, double b, int64_t n, cudaStream_t st) {
  const int nb = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  axpby_kernel<T><<<nb, 256, 0, st>>>(y, x, a, b, n);
  WC4D_LAUNCH_CHECK();
}
template void vec_axpby<double>(double*, const double*, double, double, int64_t, cudaStream_t);
template void vec_axpby<float>(float*, const float*, double, double, int64_t, cudaStream_t);

__global__ void sub_kernel(const double* a, const double* b, double* o, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    o[e] = a[e] - b[e];
}
void vec_sub(const double* a, const double* b, double* out, int64_t n, cudaStream_t st) {
  const int nb = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  sub_kernel<<<nb, 256, 0, st>>>(a, b, out, n);
  WC4D_LAUNCH_CHECK();
}

template <typename TD, typename TS>
__global__ void convert_kernel(const TS* s, TD* d, int64_t n, double scale) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    d[e] = (TD)((double)s[e] * scale);
}
template <typename TD, typename TS>
void vec_convert(const TS* src, TD* dst, int64_t n, double scale, cudaStream_t st) {
  const int nb = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  convert_kernel<TD, TS><<<nb, 256, 0, st>>>(src, dst, n, scale);
  WC4D_LAUNCH_CHECK();
}
template void vec_convert<float, double>(const double*, float*, int64_t, double, cudaStream_t);
template void vec_convert<double, float>(const float*, double*, int64_t, double, cudaStream_t);
template void vec_convert<double, double>(const double*, double*, int64_t, double, cudaStream_t);

}  // namespace wc4d
