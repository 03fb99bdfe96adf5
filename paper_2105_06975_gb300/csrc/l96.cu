// Lorenz-96 pieces of the incremental Gauss-Newton outer loop (Sec. 2.1,
// Sec. 7.1): RK4 forecasts of every assimilation window in parallel, the
// banded tangent-linear models M_t (exact Jacobians of the RK4 steps), and the
// right-hand side (b, d, 0) about the current trajectory.
//
//   dx_j/dt = (x_{j+1} - x_{j-2}) x_{j-1} - x_j + F   (periodic)
//
// One CTA owns one state vector of length s in shared memory; neighbours are
// read from shared memory after a barrier, so a window's 5 x 4 RK4 stages run
// without global-memory round trips.
#include <algorithm>

#include "common.cuh"

namespace wc4d {

__device__ __forceinline__ int pw(int j, int s) { return j < 0 ? j + s : (j >= s ? j - s : j); }

__device__ __forceinline__ double l96_f(const double* x, int j, int s, double F) {
  return (x[pw(j + 1, s)] - x[pw(j - 2, s)]) * x[pw(j - 1, s)] - x[j] + F;
}
// tangent of the right-hand side at x applied to d
__device__ __forceinline__ double l96_df(const double* x, const double* d, int j, int s) {
  const double xm1 = x[pw(j - 1, s)];
  return (d[pw(j + 1, s)] - d[pw(j - 2, s)]) * xm1 + (x[pw(j + 1, s)] - x[pw(j - 2, s)]) * d[pw(j - 1, s)] - d[j];
}

// One RK4 step of the state held in shared memory (x), optionally with its
// tangent (d).  Work arrays: xs, ds (stage inputs), ax, ad (accumulators).
template <bool TANGENT>
__device__ void rk4_step_smem(double* x, double* d, double* xs, double* ds, double* ax, double* ad, int s, double F,
                              double dt) {
  const double w[4] = {1.0, 2.0, 2.0, 1.0};
  const double h[4] = {0.5 * dt, 0.5 * dt, dt, 0.0};
  for (int j = threadIdx.x; j < s; j += blockDim.x) {
    xs[j] = x[j];
    ax[j] = 0.0;
    if (TANGENT) {
      ds[j] = d[j];
      ad[j] = 0.0;
    }
  }
  __syncthreads();
  for (int stage = 0; stage < 4; ++stage) {
    // k = f(xs) (and dk = f'(xs) ds); next stage input xs' = x + h k
    double kv[8], dkv[8];
    int cnt = 0;
    for (int j = threadIdx.x; j < s; j += blockDim.x, ++cnt) {
      kv[cnt] = l96_f(xs, j, s, F);
      if (TANGENT) dkv[cnt] = l96_df(xs, ds, j, s);
    }
    __syncthreads();
    cnt = 0;
    for (int j = threadIdx.x; j < s; j += blockDim.x, ++cnt) {
      ax[j] += w[stage] * kv[cnt];
      xs[j] = x[j] + h[stage] * kv[cnt];
      if (TANGENT) {
        ad[j] += w[stage] * dkv[cnt];
        ds[j] = d[j] + h[stage] * dkv[cnt];
      }
    }
    __syncthreads();
  }
  for (int j = threadIdx.x; j < s; j += blockDim.x) {
    x[j] = x[j] + (dt / 6.0) * ax[j];
    if (TANGENT) d[j] = d[j] + (dt / 6.0) * ad[j];
  }
  __syncthreads();
}

// out[w] = RK4^steps(in[w]) for count windows (one CTA each)
__global__ void l96_forecast_kernel(const double* in, double* out, int count, int s, double F, double dt, int steps) {
  extern __shared__ double sm[];
  double *x = sm, *xs = sm + s, *ax = sm + 2 * s;
  const int win = blockIdx.x;
  if (win >= count) return;
  for (int j = threadIdx.x; j < s; j += blockDim.x) x[j] = in[(int64_t)win * s + j];
  __syncthreads();
  for (int k = 0; k < steps; ++k) rk4_step_smem<false>(x, nullptr, xs, nullptr, ax, nullptr, s, F, dt);
  for (int j = threadIdx.x; j < s; j += blockDim.x) out[(int64_t)win * s + j] = x[j];
}

// background trajectory: traj[0] = xb, traj[t] = RK4^steps(traj[t-1]) (sequential in t)
__global__ void l96_background_kernel(const double* xb, double* traj, int N, int s, double F, double dt, int steps) {
  extern __shared__ double sm[];
  double *x = sm, *xs = sm + s, *ax = sm + 2 * s;
  for (int j = threadIdx.x; j < s; j += blockDim.x) {
    x[j] = xb[j];
    traj[j] = xb[j];
  }
  __syncthreads();
  for (int t = 1; t <= N; ++t) {
    for (int k = 0; k < steps; ++k) rk4_step_smem<false>(x, nullptr, xs, nullptr, ax, nullptr, s, F, dt);
    for (int j = threadIdx.x; j < s; j += blockDim.x) traj[(int64_t)t * s + j] = x[j];
    __syncthreads();
  }
}

// Banded TLM by coloured probing.  Column c of M_t has non-zeros only in rows
// c-hi..c+lo, so columns whose indices agree modulo m (m >= lo+hi+1, m | s)
// never share a row: one tangent integration of the probe sum_{c = r mod m} e_c
// gives every such column.  CTA (t-1, r) integrates the tangent of the
// ``steps`` RK4 steps from traj[t-1] and writes, for each row j, the single band
// entry whose column is congruent to r.
__global__ void l96_tlm_band_kernel(const double* traj, double* bands, int N, int s, int lo, int hi, int m, double F,
                                    double dt, int steps) {
  extern __shared__ double sm[];
  double *x = sm, *d = sm + s, *xs = sm + 2 * s, *ds = sm + 3 * s, *ax = sm + 4 * s, *ad = sm + 5 * s;
  const int t = blockIdx.x + 1, r = blockIdx.y;
  if (t > N || r >= m) return;
  for (int j = threadIdx.x; j < s; j += blockDim.x) {
    x[j] = traj[(int64_t)(t - 1) * s + j];
    d[j] = (j % m == r) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int k = 0; k < steps; ++k) rk4_step_smem<true>(x, d, xs, ds, ax, ad, s, F, dt);
  const int w = lo + hi + 1;
  for (int j = threadIdx.x; j < s; j += blockDim.x) {
    // offset o in [-lo, hi] with (j + o) = r (mod m)
    int o = ((r - j) % m + m) % m;  // in [0, m)
    if (o > hi) o -= m;
    if (o >= -lo && o <= hi) bands[((int64_t)(t - 1) * s + j) * w + (o + lo)] = d[j];
  }
}

// rhs = (b, d, 0): b_0 = xb - traj_0, b_t = fc_{t-1} - traj_t, d_t = y_t - traj_t[obs]
__global__ void gn_rhs_kernel(const double* xb, const double* traj, const double* fc, const double* y, const int* obs,
                              int s, int N, int p, double* rhs) {
  const int64_t ns = (int64_t)(N + 1) * s, np = (int64_t)(N + 1) * p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 2 * ns + np;
       e += (int64_t)gridDim.x * blockDim.x) {
    double v;
    if (e < ns) {
      const int t = (int)(e / s), j = (int)(e % s);
      v = (t == 0) ? xb[j] - traj[j] : fc[(int64_t)(t - 1) * s + j] - traj[e];
    } else if (e < ns + np) {
      const int64_t f = e - ns;
      const int t = (int)(f / p), r = (int)(f % p);
      v = y[f] - traj[(int64_t)t * s + obs[r]];
    } else {
      v = 0.0;
    }
    rhs[e] = v;
  }
}

static int l96_threads(int s) { return std::min(1024, std::max(32, ((s + 31) / 32) * 32)); }

void l96_forecast(const double* in, double* out, int count, int s, double F, double dt, int steps, cudaStream_t st) {
  const size_t smem = sizeof(double) * 3 * s;
  if (smem > 48 * 1024)
    WC4D_CUDA(cudaFuncSetAttribute(l96_forecast_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  l96_forecast_kernel<<<count, l96_threads(s), smem, st>>>(in, out, count, s, F, dt, steps);
  WC4D_LAUNCH_CHECK();
}

void l96_background(const double* xb, double* traj, int N, int s, double F, double dt, int steps, cudaStream_t st) {
  const size_t smem = sizeof(double) * 3 * s;
  if (smem > 48 * 1024)
    WC4D_CUDA(cudaFuncSetAttribute(l96_background_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  l96_background_kernel<<<1, l96_threads(s), smem, st>>>(xb, traj, N, s, F, dt, steps);
  WC4D_LAUNCH_CHECK();
}

// colour count: the smallest divisor of s not below the band width
int l96_colors(int s, int width) {
  for (int m = width; m <= s; ++m)
    if (s % m == 0) return m;
  return s;
}

void l96_tlm_bands(const double* traj, double* bands, int N, int s, int lo, int hi, double F, double dt, int steps,
                   cudaStream_t st) {
  if (N == 0) return;
  const int m = l96_colors(s, lo + hi + 1);
  const size_t smem = sizeof(double) * 6 * s;
  if (smem > 48 * 1024)
    WC4D_CUDA(cudaFuncSetAttribute(l96_tlm_band_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  l96_tlm_band_kernel<<<dim3(N, m), l96_threads(s), smem, st>>>(traj, bands, N, s, lo, hi, m, F, dt, steps);
  WC4D_LAUNCH_CHECK();
}

void gn_rhs(const double* xb, const double* traj, const double* fc, const double* y, const int* obs, int s, int N,
            int p, double* rhs, cudaStream_t st) {
  const int64_t n = (int64_t)(2 * s + p) * (N + 1);
  gn_rhs_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, st>>>(xb, traj, fc, y, obs, s, N, p, rhs);
  WC4D_LAUNCH_CHECK();
}

}  // namespace wc4d
