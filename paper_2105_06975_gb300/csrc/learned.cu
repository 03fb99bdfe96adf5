// Kernels of the learned Schur-block correction (see learned.cuh): FP32
// periodic convolutions with their data and weight gradients, the relative
// squared-error loss, Adam, and a counter-based normal generator for the
// training draws.  Channel counts are small (N+1 time levels, <= 64 hidden),
// so the convolutions run on the FP32 pipe from shared-memory tiles: a block
// takes 128 grid points x 8 output channels, stages the input tile (with its
// 2-point periodic halo) and the weights, and every thread accumulates one
// grid point for the 8 channels.
#include <algorithm>

#include "learned.cuh"

namespace wc4d {

constexpr int CV_X = 128;      // grid points per block (one per thread)
constexpr int CV_CO = 8;       // output channels per block
constexpr int CV_CIMAX = 64;   // input channels staged at once
constexpr int WG_X = 64;       // grid points per tile of the weight gradient
constexpr int WG_P = 4;        // (co, ci) pairs per thread per pass of the weight gradient

// out[b][co][x] = bias[co] + sum_ci sum_k Weff[co][ci][k] in[b][ci][(x + k - 2) mod s]
// flip = 0: Weff = W[co][ci][k] (W stored [Co][Ci][5]);
// flip = 1: Weff = W[ci][co][4 - k] (W stored [Ci][Co][5]) -- the data gradient.
// relu: max(., 0); mask (nullable): out *= (mask[b][co][x] > 0).
__global__ void __launch_bounds__(CV_X) conv_kernel(const float* __restrict__ in, int Ci, const float* __restrict__ W,
                                                    const float* __restrict__ bias, int Co, int s, int flip, int relu,
                                                    const float* __restrict__ mask, float* __restrict__ out) {
  __shared__ float tile[CV_CIMAX][CV_X + NET_KW - 1];
  __shared__ float ws[CV_CO][CV_CIMAX][NET_KW];
  const int x0 = blockIdx.x * CV_X, co0 = blockIdx.y * CV_CO, b = blockIdx.z;
  const float* inb = in + (int64_t)b * Ci * s;
  for (int e = threadIdx.x; e < Ci * (CV_X + NET_KW - 1); e += blockDim.x) {
    const int ci = e / (CV_X + NET_KW - 1), xx = e % (CV_X + NET_KW - 1);
    const int x = x0 + xx - NET_KW / 2;  // periodic: -2 .. s + CV_X wrap into [0, s)
    tile[ci][xx] = inb[(int64_t)ci * s + ((x % s) + s) % s];
  }
  for (int e = threadIdx.x; e < CV_CO * Ci * NET_KW; e += blockDim.x) {
    const int c = e / (Ci * NET_KW), r = e % (Ci * NET_KW), ci = r / NET_KW, k = r % NET_KW;
    const int co = co0 + c;
    float w = 0.f;
    if (co < Co) w = flip ? W[((int64_t)ci * Co + co) * NET_KW + (NET_KW - 1 - k)] : W[((int64_t)co * Ci + ci) * NET_KW + k];
    ws[c][ci][k] = w;
  }
  __syncthreads();
  const int x = x0 + threadIdx.x;
  if (x >= s) return;
  float acc[CV_CO];
#pragma unroll
  for (int c = 0; c < CV_CO; ++c) acc[c] = (bias && co0 + c < Co) ? bias[co0 + c] : 0.f;
  for (int ci = 0; ci < Ci; ++ci) {
    float v[NET_KW];
#pragma unroll
    for (int k = 0; k < NET_KW; ++k) v[k] = tile[ci][threadIdx.x + k];
#pragma unroll
    for (int c = 0; c < CV_CO; ++c)
#pragma unroll
      for (int k = 0; k < NET_KW; ++k) acc[c] = fmaf(ws[c][ci][k], v[k], acc[c]);
  }
#pragma unroll
  for (int c = 0; c < CV_CO; ++c) {
    const int co = co0 + c;
    if (co >= Co) break;
    float r = acc[c];
    if (relu) r = fmaxf(r, 0.f);
    const int64_t o = ((int64_t)b * Co + co) * s + x;
    if (mask && !(mask[o] > 0.f)) r = 0.f;
    out[o] = r;
  }
}

static void conv(const float* in, int Ci, const float* W, const float* bias, int Co, int s, int B, int flip, int relu,
                 const float* mask, float* out, cudaStream_t st) {
  WC4D_CHECK(Ci <= CV_CIMAX, WC4D_ERR_ARG, "learned net: at most 64 input channels");
  dim3 grid((s + CV_X - 1) / CV_X, (Co + CV_CO - 1) / CV_CO, B);
  conv_kernel<<<grid, CV_X, 0, st>>>(in, Ci, W, bias, Co, s, flip, relu, mask, out);
  WC4D_LAUNCH_CHECK();
}

void net_forward(const NetShape& sh, const float* params, int B, const float* in, float* const acts[3], float* out,
                 cudaStream_t st) {
  const float* h = in;
  for (int l = 0; l < NET_LAYERS; ++l) {
    float* o = (l < NET_LAYERS - 1) ? acts[l] : out;
    conv(h, sh.ci(l), params + sh.w_off(l), params + sh.b_off(l), sh.co(l), sh.s, B, 0, l < NET_LAYERS - 1, nullptr,
         o, st);
    h = o;
  }
}

// one block per sample: gout = 2 (in + out - tn) / (tn2 B), loss += |in + out - tn|^2 / tn2
__global__ void loss_grad_kernel(const float* in, const float* out, const float* tn, const double* tn2,
                                 const int* idx, float* gout, double* loss_sum, int64_t len, int B) {
  __shared__ double sh[32];
  const int b = blockIdx.x;
  const double inv = 1.0 / fmax(tn2[idx ? idx[b] : b], 1e-300);
  const float scale = (float)(2.0 * inv / B);
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < len; e += blockDim.x) {
    const int64_t o = (int64_t)b * len + e;
    const float d = in[o] + out[o] - tn[o];
    gout[o] = scale * d;
    acc += (double)d * d;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) atomicAdd(loss_sum, acc * inv);
}

void net_loss_grad(const NetShape& sh, int B, const float* in, const float* out, const float* tn, const double* tn2,
                   const int* idx, float* gout, double* loss_sum, cudaStream_t st) {
  loss_grad_kernel<<<B, 256, 0, st>>>(in, out, tn, tn2, idx, gout, loss_sum, (int64_t)sh.C * sh.s, B);
  WC4D_LAUNCH_CHECK();
}

// Weight / bias gradient partials of one layer, one block per sample:
// part[b][(co*Ci + ci)*5 + k] = sum_x g[b][co][x] in[b][ci][(x + k - 2) mod s],
// part[b][Co*Ci*5 + co] = sum_x g[b][co][x].
__global__ void __launch_bounds__(256) wgrad_kernel(const float* __restrict__ in, int Ci,
                                                    const float* __restrict__ g, int Co, int s,
                                                    float* __restrict__ part) {
  __shared__ float ti[CV_CIMAX][WG_X + NET_KW - 1];
  __shared__ float tg[CV_CIMAX][WG_X];
  const int b = blockIdx.x;
  const float* inb = in + (int64_t)b * Ci * s;
  const float* gb = g + (int64_t)b * Co * s;
  const int npair = Co * Ci + Co;
  const int64_t stride = (int64_t)Co * Ci * NET_KW + Co;
  float* pb = part + (int64_t)b * stride;
  // each thread owns pairs p = pbase + tid + 256 q (q < WG_P), sums in registers;
  // the sample's tiles are re-read (from L2) once per pass
  for (int pbase = 0; pbase < npair; pbase += 256 * WG_P) {
    float acc[WG_P][NET_KW];
#pragma unroll
    for (int q = 0; q < WG_P; ++q)
#pragma unroll
      for (int k = 0; k < NET_KW; ++k) acc[q][k] = 0.f;
    for (int x0 = 0; x0 < s; x0 += WG_X) {
      __syncthreads();
      for (int e = threadIdx.x; e < Ci * (WG_X + NET_KW - 1); e += blockDim.x) {
        const int ci = e / (WG_X + NET_KW - 1), xx = e % (WG_X + NET_KW - 1);
        const int x = x0 + xx - NET_KW / 2;
        ti[ci][xx] = inb[(int64_t)ci * s + (((x % s) + s) % s)];
      }
      for (int e = threadIdx.x; e < Co * WG_X; e += blockDim.x) {
        const int co = e / WG_X, xx = e % WG_X;
        tg[co][xx] = (x0 + xx < s) ? gb[(int64_t)co * s + x0 + xx] : 0.f;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < WG_P; ++q) {
        const int p = pbase + threadIdx.x + 256 * q;
        if (p >= npair) continue;
        if (p < Co * Ci) {
          const int co = p / Ci, ci = p % Ci;
          for (int xx = 0; xx < WG_X; ++xx) {
            const float gv = tg[co][xx];
#pragma unroll
            for (int k = 0; k < NET_KW; ++k) acc[q][k] = fmaf(gv, ti[ci][xx + k], acc[q][k]);
          }
        } else {
          const int co = p - Co * Ci;
          for (int xx = 0; xx < WG_X; ++xx) acc[q][0] += tg[co][xx];
        }
      }
    }
#pragma unroll
    for (int q = 0; q < WG_P; ++q) {
      const int p = pbase + threadIdx.x + 256 * q;
      if (p >= npair) continue;
      if (p < Co * Ci) {
#pragma unroll
        for (int k = 0; k < NET_KW; ++k) pb[(int64_t)p * NET_KW + k] = acc[q][k];
      } else {
        pb[(int64_t)Co * Ci * NET_KW + (p - Co * Ci)] = acc[q][0];
      }
    }
  }
}

// grads[j] = sum_b part[b][j] (fixed order)
__global__ void part_sum_kernel(const float* part, int B, int64_t stride, float* out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < stride; j += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < B; ++b) acc += part[(int64_t)b * stride + j];
    out[j] = (float)acc;
  }
}

int64_t net_wpart_elems(const NetShape& sh, int B) {
  int64_t m = 0;
  for (int l = 0; l < NET_LAYERS; ++l) m = std::max<int64_t>(m, (int64_t)sh.co(l) * sh.ci(l) * NET_KW + sh.co(l));
  return m * B;
}

void net_backward(const NetShape& sh, const float* params, int B, const float* in, float* const acts[3],
                  const float* gout, float* grads, float* scratch0, float* scratch1, float* wpart, int64_t wpart_cap,
                  cudaStream_t st) {
  WC4D_CHECK(net_wpart_elems(sh, B) <= wpart_cap, WC4D_ERR_ARG, "learned net: gradient partial buffer too small");
  const float* g = gout;
  float* bufs[2] = {scratch0, scratch1};
  for (int l = NET_LAYERS - 1; l >= 0; --l) {
    const float* lin = (l == 0) ? in : acts[l - 1];
    const int Ci = sh.ci(l), Co = sh.co(l);
    wgrad_kernel<<<B, 256, 0, st>>>(lin, Ci, g, Co, sh.s, wpart);
    WC4D_LAUNCH_CHECK();
    const int64_t stride = (int64_t)Co * Ci * NET_KW + Co;
    part_sum_kernel<<<(int)std::min<int64_t>((stride + 255) / 256, 152 * 4), 256, 0, st>>>(wpart, B, stride,
                                                                                         grads + sh.w_off(l));
    WC4D_LAUNCH_CHECK();
    if (l > 0) {
      // data gradient through conv l, then the ReLU of layer l-1 (mask = its output > 0)
      float* gin = bufs[l & 1];
      conv(g, Co, params + sh.w_off(l), nullptr, Ci, sh.s, B, 1, 0, acts[l - 1], gin, st);
      g = gin;
    }
  }
}

__global__ void adam_kernel(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                            float c1, float c2, float eps) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

void net_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, int t, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  adam_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 4), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, c1, c2,
                                                                                1e-8f);
  WC4D_LAUNCH_CHECK();
}

__global__ void gather_kernel(const float* src, const int* idx, int B, int64_t len, float* dst) {
  const int b = blockIdx.y;
  const float* sp = src + (int64_t)idx[b] * len;
  float* dp = dst + (int64_t)b * len;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x)
    dp[e] = sp[e];
}

void net_gather(const float* src, const int* idx, int B, int64_t len, float* dst, cudaStream_t st) {
  dim3 grid((unsigned)std::min<int64_t>((len + 255) / 256, 64), B);
  gather_kernel<<<grid, 256, 0, st>>>(src, idx, B, len, dst);
  WC4D_LAUNCH_CHECK();
}

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) of seed + counter as the
// uniform source; Box-Muller for the normal pair of counters (2i, 2i+1).
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void normal_kernel(double* out, int64_t n, uint64_t seed, uint64_t base) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t c = 2 * (base + (uint64_t)i);
    const uint64_t a = splitmix64(seed * 0x632BE59BD9B4E019ull + c);
    const uint64_t b = splitmix64(seed * 0x632BE59BD9B4E019ull + c + 1);
    const float u1 = ((float)(a >> 40) + 1.0f) * (1.0f / 16777216.0f);  // (0, 1]
    const float u2 = (float)(b >> 40) * (1.0f / 16777216.0f);           // [0, 1)
    out[i] = (double)(sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2));
  }
}

void normal_fill(double* out, int64_t n, uint64_t seed, uint64_t base, cudaStream_t st) {
  normal_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, st>>>(out, n, seed, base);
  WC4D_LAUNCH_CHECK();
}

__global__ void in_from_kernel(const double* y, const double* nrm2, float* yn, int64_t n) {
  const double nrm = sqrt_clamped(*nrm2);
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    yn[e] = (float)(y[e] * inv);
}
void net_in_from(const double* y, const double* nrm2, float* yn, int64_t n, cudaStream_t st) {
  in_from_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, st>>>(y, nrm2, yn, n);
  WC4D_LAUNCH_CHECK();
}

__global__ void out_to_kernel(const float* yn, const float* f, const double* nrm2, double* z, int64_t n) {
  const double nrm = sqrt_clamped(*nrm2);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    z[e] = nrm * ((double)yn[e] + (double)f[e]);
}
void net_out_to(const float* yn, const float* f, const double* nrm2, double* z, int64_t n, cudaStream_t st) {
  out_to_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, st>>>(yn, f, nrm2, z, n);
  WC4D_LAUNCH_CHECK();
}

// d = yn + f - tn (f may be NULL: the plain block) as doubles
__global__ void resid_kernel(const float* yn, const float* f, const float* tn, double* d, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    d[e] = (double)yn[e] + (f ? (double)f[e] : 0.0) - (double)tn[e];
}
void net_resid(const float* yn, const float* f, const float* tn, double* d, int64_t n, cudaStream_t st) {
  resid_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, st>>>(yn, f, tn, d, n);
  WC4D_LAUNCH_CHECK();
}

__global__ void store_pair_kernel(const double* y, const double* t, const double* nrm2, float* yn, float* tn,
                                  double* tn2_acc, int64_t n) {
  __shared__ double sh[32];
  const double nrm = sqrt_clamped(*nrm2);
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    yn[e] = (float)(y[e] * inv);
    const float tv = (float)(t[e] * inv);
    tn[e] = tv;
    acc += (double)tv * tv;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) atomicAdd(tn2_acc, acc);
}
void net_store_pair(const double* y, const double* t, const double* nrm2, float* yn, float* tn, double* tn2_acc,
                    int64_t n, cudaStream_t st) {
  store_pair_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 2), 256, 0, st>>>(y, t, nrm2, yn, tn, tn2_acc, n);
  WC4D_LAUNCH_CHECK();
}

}  // namespace wc4d
