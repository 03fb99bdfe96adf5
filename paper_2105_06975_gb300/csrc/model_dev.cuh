// Device-side application of the model matrices M_t and M_t^T at one grid point.
#pragma once
#include "common.cuh"

namespace wc4d {

__device__ __forceinline__ int wrap_idx(int j, int s) {
  j += (j < 0) ? s : 0;
  j -= (j >= s) ? s : 0;
  return j;
}

// (M_t x)_j, t = 1..N  (Eq. def:L: block row t carries -M_t)
template <typename T>
__device__ __forceinline__ T model_apply(const ModelDev& md, int t, const T* __restrict__ x, int j) {
  const int s = md.s;
  if (md.kind == WC4D_MODEL_STENCIL3) {
    const int jm = (j == 0) ? s - 1 : j - 1;
    const int jp = (j == s - 1) ? 0 : j + 1;
    return T(md.c0) * x[jm] + T(md.c1) * x[j] + T(md.c2) * x[jp];
  }
  const int w = md.lo + md.hi + 1;
  const double* b = md.bands + ((int64_t)(t - 1) * s + j) * w;
  T acc = T(0);
  for (int o = -md.lo; o <= md.hi; ++o) acc += T(b[o + md.lo]) * x[wrap_idx(j + o, s)];
  return acc;
}

// (M_t^T y)_j
template <typename T>
__device__ __forceinline__ T model_apply_T(const ModelDev& md, int t, const T* __restrict__ y, int j) {
  const int s = md.s;
  if (md.kind == WC4D_MODEL_STENCIL3) {
    const int jm = (j == 0) ? s - 1 : j - 1;
    const int jp = (j == s - 1) ? 0 : j + 1;
    return T(md.c0) * y[jp] + T(md.c1) * y[j] + T(md.c2) * y[jm];
  }
  const int w = md.lo + md.hi + 1;
  const double* b = md.bands + (int64_t)(t - 1) * s * w;
  T acc = T(0);
  for (int o = -md.lo; o <= md.hi; ++o) {
    const int i = wrap_idx(j - o, s);  // row i of M_t holds column j at offset o
    acc += T(b[(int64_t)i * w + o + md.lo]) * y[i];
  }
  return acc;
}

}  // namespace wc4d
