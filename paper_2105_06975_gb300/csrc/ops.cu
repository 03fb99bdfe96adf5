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
  pdl_wait();
  pdl_trigger();
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

// The same sweep with each chunk's grid cut into segments of W points, one CTA
// per (chunk, segment): a CTA starts from the chunk's first level on its
// segment widened by R (k-1) points on each side (R = the model's reach, 1 for
// the 3-point stencil, max(lo, hi) for bands; periodic), keeps the running level
// in shared memory and narrows the valid range by R per step, so no CTA needs
// another's values.  Every output element is computed with the same operations
// in the same order as lhat_sweep_kernel.  Needs v and z not to overlap.
template <typename T>
__device__ __forceinline__ T local_apply(const ModelDev& md, int t, const T* cur, int e, int x, bool transpose) {
  const int s = md.s;
  if (md.kind == WC4D_MODEL_STENCIL3) {
    return transpose ? T(md.c0) * cur[e + 1] + T(md.c1) * cur[e] + T(md.c2) * cur[e - 1]
                     : T(md.c0) * cur[e - 1] + T(md.c1) * cur[e] + T(md.c2) * cur[e + 1];
  }
  const int w = md.lo + md.hi + 1;
  T acc = T(0);
  if (!transpose) {
    const double* b = md.bands + ((int64_t)(t - 1) * s + x) * w;
    for (int o = -md.lo; o <= md.hi; ++o) acc += T(b[o + md.lo]) * cur[e + o];
  } else {
    const double* b = md.bands + (int64_t)(t - 1) * s * w;
    for (int o = -md.lo; o <= md.hi; ++o) {
      const int i = wrap_idx(x - o, s);
      acc += T(b[(int64_t)i * w + o + md.lo]) * cur[e - o];
    }
  }
  return acc;
}

template <typename T>
__global__ void __launch_bounds__(256) lhat_sweep_seg_kernel(ModelDev md, int k, const T* __restrict__ v,
                                                             T* __restrict__ z, int transpose, int identity_model,
                                                             int W, int R, const int* done) {
  pdl_wait();
  pdl_trigger();
  if (done != nullptr && *(volatile const int*)done) return;
  extern __shared__ unsigned char smraw[];
  T* bufA = reinterpret_cast<T*>(smraw);
  const int s = md.s, T1 = md.N + 1;
  const int t0 = blockIdx.x * k, t1 = min(t0 + k, T1) - 1, steps = t1 - t0;
  const int x0 = blockIdx.y * W, x1 = min(x0 + W, s);
  const int H = R * steps, E = (x1 - x0) + 2 * H;
  T* bufB = bufA + E;
  auto gx = [&](int e) { return wrap_idx(x0 - H + e, s); };
  const int ts = transpose ? t1 : t0;
  for (int e = threadIdx.x; e < E; e += blockDim.x) {
    const T val = v[(int64_t)ts * s + gx(e)];
    bufA[e] = val;
    if (e >= H && e < H + (x1 - x0)) z[(int64_t)ts * s + gx(e)] = val;
  }
  __syncthreads();
  T* cur = bufA;
  T* nxt = bufB;
  for (int m = 1; m <= steps; ++m) {
    const int t = transpose ? t1 - m : t0 + m;   // level being formed
    const int tm = transpose ? t + 1 : t;        // forward uses M_t on z_{t-1}; transpose M_{t+1}^T on z_{t+1}
    const int lo_e = R * m, hi_e = E - R * m;
    for (int e = lo_e + threadIdx.x; e < hi_e; e += blockDim.x) {
      const int x = gx(e);
      const T mz = identity_model ? cur[e] : local_apply<T>(md, tm, cur, e, x, transpose != 0);
      const T val = v[(int64_t)t * s + x] + mz;
      nxt[e] = val;
      if (e >= H && e < H + (x1 - x0)) z[(int64_t)t * s + x] = val;
    }
    __syncthreads();
    T* tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
}

template <typename T>
void lhat_sweep(const ModelDev& md, int k, const T* v, T* z, bool transpose, bool identity_model, const int* done,
                cudaStream_t st) {
  const int nchunks = (md.N + 1 + k - 1) / k;
  const int s = md.s;
  const int R = identity_model ? 0 : (md.kind == WC4D_MODEL_STENCIL3 ? 1 : std::max(md.lo, md.hi));
  const int steps = std::min(k, md.N + 1) - 1;
  // about two CTAs per SM over (chunks x segments); segments of >= 128 points
  int nseg = std::max(1, (152 * 2) / nchunks);
  int W = ((s + nseg - 1) / nseg + 31) / 32 * 32;
  W = std::max(W, 128);
  nseg = (s + W - 1) / W;
  const int E = W + 2 * R * steps;
  const bool alias = (const void*)v == (const void*)z;
  if (nseg > 1 && !alias && steps > 0 && 2 * R * steps <= W && E <= s &&
      (size_t)E * 2 * sizeof(T) <= 48 * 1024) {
    WC4D_CUDA(launch_pdl(lhat_sweep_seg_kernel<T>, dim3(nchunks, nseg), dim3(256), (size_t)E * 2 * sizeof(T), st, md, k,
                         v, z, transpose ? 1 : 0, identity_model ? 1 : 0, W, R, done));
    WC4D_LAUNCH_CHECK();
    return;
  }
  const int threads = std::min(1024, ((md.s + 31) / 32) * 32);
  WC4D_CUDA(launch_pdl(lhat_sweep_kernel<T>, dim3(nchunks), dim3(threads), 0, st, md, k, v, z, transpose ? 1 : 0,
                       identity_model ? 1 : 0, done));
  WC4D_LAUNCH_CHECK();
}
template void lhat_sweep<double>(const ModelDev&, int, const double*, double*, bool, bool, const int*, cudaStream_t);
template void lhat_sweep<float>(const ModelDev&, int, const float*, float*, bool, bool, const int*, cudaStream_t);

void launch_lhat_sweep(const ModelDev& md, int k, const double* v, double* z, bool transpose, bool identity_model,
                       const int* done, cudaStream_t st) {
  lhat_sweep<double>(md, k, v, z, transpose, identity_model, done, st);
}

// c3_t[j] = v1_t[j] - [t < N] (M_{t+1}^T v1_{t+1})[j] + (H_t^T v2_t)[j],
// H_t^T scatters nu_t[r] to grid point obs_t[r]; inv[t * inv_stride + j] = r or
// -1 (inv_stride = 0: one set for every time, nu_t at t p; inv_stride = s:
// per-time sets, nu_t at nuoff[t]).
// c3h / c3l (optional): the double-float split of c3 (hi = round(c3), lo = round(c3 - hi))
template <typename T>
__global__ void saddle_c3_kernel(ModelDev md, const T* __restrict__ v1, const T* __restrict__ v2,
                                 const int* __restrict__ inv, int p, T* __restrict__ c3, float* __restrict__ c3h,
                                 float* __restrict__ c3l, const int* done, int inv_stride = 0,
                                 const int* __restrict__ nuoff = nullptr) {
  pdl_wait();
  pdl_trigger();
  if (done != nullptr && *(volatile const int*)done) return;
  const int s = md.s, N = md.N;
  const int64_t total = (int64_t)(N + 1) * s;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int t, j;
    idx_divmod(e, s, total < ((int64_t)1 << 31), t, j);
    T val = v1[e];
    if (t < N) val -= model_apply_T<T>(md, t + 1, v1 + (int64_t)(t + 1) * s, j);
    const int r = inv[(int64_t)t * inv_stride + j];
    if (r >= 0) val += v2[(nuoff ? (int64_t)nuoff[t] : (int64_t)t * p) + r];
    c3[e] = val;
    if (c3h != nullptr) {
      const float h = (float)val;
      c3h[e] = h;
      c3l[e] = (float)((double)val - (double)h);
    }
  }
}

template <typename T>
void saddle_c3(const ModelDev& md, const T* v1, const T* v2, const int* inv, int p, T* c3, const int* done,
               cudaStream_t st) {
  const int64_t total = (int64_t)(md.N + 1) * md.s;
  const int nb = (int)std::min<int64_t>((total + 255) / 256, 152 * 8);
  WC4D_CUDA(launch_pdl(saddle_c3_kernel<T>, dim3(nb), dim3(256), 0, st, md, v1, v2, inv, p, c3, (float*)nullptr,
                       (float*)nullptr, done, 0, (const int*)nullptr));
  WC4D_LAUNCH_CHECK();
}
void saddle_c3_split(const ModelDev& md, const double* v1, const double* v2, const int* inv, int p, double* c3,
                     float* c3h, float* c3l, const int* done, cudaStream_t st) {
  const int64_t total = (int64_t)(md.N + 1) * md.s;
  const int nb = (int)std::min<int64_t>((total + 255) / 256, 152 * 8);
  WC4D_CUDA(launch_pdl(saddle_c3_kernel<double>, dim3(nb), dim3(256), 0, st, md, v1, v2, inv, p, c3, c3h, c3l, done,
                       0, (const int*)nullptr));
  WC4D_LAUNCH_CHECK();
}
void saddle_c3_pertime(const ModelDev& md, const double* v1, const double* v2, const int* inv_all, const int* nuoff,
                       double* c3, float* c3h, float* c3l, const int* done, cudaStream_t st) {
  const int64_t total = (int64_t)(md.N + 1) * md.s;
  const int nb = (int)std::min<int64_t>((total + 255) / 256, 152 * 8);
  WC4D_CUDA(launch_pdl(saddle_c3_kernel<double>, dim3(nb), dim3(256), 0, st, md, v1, v2, inv_all, 0, c3, c3h, c3l,
                       done, md.s, nuoff));
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
