// Time-direction operators: the Lhat = L_M(k) sweeps (Definition 1, Lemma 1)
// and the third block row of A v (c3 = L^T v1 + H^T v2, Sec. 6.2).
#include <algorithm>

#include "common.cuh"
#include "model_dev.cuh"

namespace wc4d {

// One CTA per chunk of L_M(k): time levels {c k, ..., min((c+1) k, N+1) - 1}.
// Forward (Lhat^{-1}):   z_{t0} = v_{t0},  z_t = v_t + M_t z_{t-1}.
// Transpose (Lhat^{-T}): z_{t1} = v_{t1},  z_t = v_t + M_{t+1}^T z_{t+1}.
// identity_model: every M_t replaced by I (L_I of Sec. 2.2).
// z may alias v (each step reads only the previous level of z and its own v).
template <typename T>
__global__ void __launch_bounds__(1024) lhat_sweep_kernel(ModelDev md, int k, const T* v, T* z, int transpose,
                                                          int identity_model, const int* done) {
  if (done != nullptr && *(volatile const int*)done) return;
  const int s = md.s, T1 = md.N + 1;
  const int t0 = blockIdx.x * k;
  const int t1 = min(t0 + k, T1) - 1;
  if (!transpose) {
    for (int j = threadIdx.x; j < s; j += blockDim.x) z[(int64_t)t0 * s + j] = v[(int64_t)t0 * s + j];
    __syncthreads();
    for (int t = t0 + 1; t <= t1; ++t) {
      const T* zp = z + (int64_t)(t - 1) * s;
      for (int j = threadIdx.x; j < s; j += blockDim.x) {
        const T mz = identity_model ? zp[j] : model_apply<T>(md, t, zp, j);
        z[(int64_t)t * s + j] = v[(int64_t)t * s + j] + mz;
      }
      __syncthreads();
    }
  } else {
    for (int j = threadIdx.x; j < s; j += blockDim.x) z[(int64_t)t1 * s + j] = v[(int64_t)t1 * s + j];
    __syncthreads();
    for (int t = t1 - 1; t >= t0; --t) {
      const T* zn = z + (int64_t)(t + 1) * s;
      for (int j = threadIdx.x; j < s; j += blockDim.x) {
        const T mz = identity_model ? zn[j] : model_apply_T<T>(md, t + 1, zn, j);
        z[(int64_t)t * s + j] = v[(int64_t)t * s + j] + mz;
      }
      __syncthreads();
    }
  }
}

template <typename T>
void lhat_sweep(const ModelDev& md, int k, const T* v, T* z, bool transpose, bool identity_model, const int* done,
                cudaStream_t st) {
  const int nchunks = (md.N + 1 + k - 1) / k;
  const int threads = std::min(1024, ((md.s + 31) / 32) * 32);
  lhat_sweep_kernel<T><<<nchunks, threads, 0, st>>>(md, k, v, z, transpose ? 1 : 0, identity_model ? 1 : 0, done);
  WC4D_LAUNCH_CHECK();
}
template void lhat_sweep<double>(const ModelDev&, int, const double*, double*, bool, bool, const int*, cudaStream_t);
template void lhat_sweep<float>(const ModelDev&, int, const float*, float*, bool, bool, const int*, cudaStream_t);

void launch_lhat_sweep(const ModelDev& md, int k, const double* v, double* z, bool transpose, bool identity_model,
                       const int* done, cudaStream_t st) {
  lhat_sweep<double>(md, k, v, z, transpose, identity_model, done, st);
}

// c3_t[j] = v1_t[j] - [t < N] (M_{t+1}^T v1_{t+1})[j] + (H^T v2_t)[j],
// H^T scatters nu_t[r] to grid point obs[r]; inv[j] = r or -1.
template <typename T>
__global__ void saddle_c3_kernel(ModelDev md, const T* __restrict__ v1, const T* __restrict__ v2,
                                 const int* __restrict__ inv, int p, T* __restrict__ c3, const int* done) {
  if (done != nullptr && *(volatile const int*)done) return;
  const int s = md.s, N = md.N;
  const int64_t total = (int64_t)(N + 1) * s;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(e / s), j = (int)(e % s);
    T val = v1[e];
    if (t < N) val -= model_apply_T<T>(md, t + 1, v1 + (int64_t)(t + 1) * s, j);
    const int r = inv[j];
    if (r >= 0) val += v2[(int64_t)t * p + r];
    c3[e] = val;
  }
}

template <typename T>
void saddle_c3(const ModelDev& md, const T* v1, const T* v2, const int* inv, int p, T* c3, const int* done,
               cudaStream_t st) {
  const int64_t total = (int64_t)(md.N + 1) * md.s;
  const int nb = (int)std::min<int64_t>((total + 255) / 256, 152 * 8);
  saddle_c3_kernel<T><<<nb, 256, 0, st>>>(md, v1, v2, inv, p, c3, done);
  WC4D_LAUNCH_CHECK();
}
template void saddle_c3<double>(const ModelDev&, const double*, const double*, const int*, int, double*, const int*,
                                cudaStream_t);
template void saddle_c3<float>(const ModelDev&, const float*, const float*, const int*, int, float*, const int*,
                               cudaStream_t);

void launch_saddle_c3(const ModelDev& md, const double* v1, const double* v2, const int* inv, int p, double* c3,
                      const int* done, cudaStream_t st) {
  saddle_c3<double>(md, v1, v2, inv, p, c3, done, st);
}

}  // namespace wc4d
