// Learned Schur-block correction (not in the paper): a 1D convolutional
// network over the grid with the N+1 time levels as channels.
//   z = |y| (yn + f(yn)),  yn = y / |y|,  y = S_hat^{-1} r  (third block of P_D)
// f: conv(C->H) ReLU conv(H->H) ReLU conv(H->H) ReLU conv(H->C), kernel 5,
// periodic 'same' padding; tap k reads position (x + k - 2) mod s.
// Parameters, one flat FP32 array: layer l stores W[co][ci][5] then b[co].
#pragma once
#include "common.cuh"

namespace wc4d {

constexpr int NET_KW = 5;
constexpr int NET_LAYERS = 4;

struct NetShape {
  int C = 0, H = 0, s = 0;
  int ci(int l) const { return l == 0 ? C : H; }
  int co(int l) const { return l == NET_LAYERS - 1 ? C : H; }
  int64_t w_off(int l) const {
    int64_t o = 0;
    for (int i = 0; i < l; ++i) o += (int64_t)co(i) * ci(i) * NET_KW + co(i);
    return o;
  }
  int64_t b_off(int l) const { return w_off(l) + (int64_t)co(l) * ci(l) * NET_KW; }
  int64_t nparams() const { return w_off(NET_LAYERS); }
  int64_t act_elems(int B) const { return (int64_t)B * H * s; }
};

// Forward for B samples: in [B][C][s] (normalised), acts[l] [B][co(l)][s] for
// l = 0..2 (post-ReLU), out [B][C][s] = f(in).
void net_forward(const NetShape& sh, const float* params, int B, const float* in, float* const acts[3], float* out,
                 cudaStream_t st);
// Loss |in + out - tn|^2 / tn2 per sample (tn2 = |tn|^2, indexed through idx
// when idx is not NULL), summed into loss_sum (device, one double);
// gout = d(mean loss)/d out.
void net_loss_grad(const NetShape& sh, int B, const float* in, const float* out, const float* tn, const double* tn2,
                   const int* idx, float* gout, double* loss_sum, cudaStream_t st);
// Backward: given gout = d loss / d out, accumulate parameter gradients into
// grads (overwritten).  scratch: 2 x [B][max(C,H)][s] floats; wpart: partials.
void net_backward(const NetShape& sh, const float* params, int B, const float* in, float* const acts[3],
                  const float* gout, float* grads, float* scratch0, float* scratch1, float* wpart, int64_t wpart_cap,
                  cudaStream_t st);
int64_t net_wpart_elems(const NetShape& sh, int B);
// Adam step on n parameters (bias-corrected; t = step count from 1).
void net_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, int t, cudaStream_t st);
// Gather rows idx[0..B) of src [num][len] into dst [B][len].
void net_gather(const float* src, const int* idx, int B, int64_t len, float* dst, cudaStream_t st);
// Standard normal doubles from a counter-based generator (SplitMix64 of
// seed + counter, Box-Muller): out[i] for counters base .. base+n-1.
void normal_fill(double* out, int64_t n, uint64_t seed, uint64_t base, cudaStream_t st);
// y (double) -> yn = y / |y| (float), |y| from nrm2 (device, |y|^2);
// and back: z = |y| (yn + f) as double.
void net_in_from(const double* y, const double* nrm2, float* yn, int64_t n, cudaStream_t st);
void net_out_to(const float* yn, const float* f, const double* nrm2, double* z, int64_t n, cudaStream_t st);
// d = yn + f - tn in double (f NULL: yn - tn)
void net_resid(const float* yn, const float* f, const float* tn, double* d, int64_t n, cudaStream_t st);
// Training pair store: yn = y / |y|, tn = t / |y| (float), tn2 = |tn|^2.
void net_store_pair(const double* y, const double* t, const double* nrm2, float* yn, float* tn, double* tn2_acc,
                    int64_t n, cudaStream_t st);

}  // namespace wc4d
