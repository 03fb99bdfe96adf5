// Per-time R-family products (Sec. 2.1: R = blkdiag(R_0..R_N) with R_i over
// time i's own observed points): out_t = op(A_t) x_t for every time level in
// one launch.  Each operator entry is read once for one multiply-add, so the
// kernel is a batched GEMV bound by HBM (or, in FP64, by the FP64 pipe near
// 0.7 of the HBM rate).  A CTA takes 32 rows of one time level, 4 per warp;
// the lanes stride along k (the contiguous index of the "TN" form), so every
// warp load is a 256-byte coalesced segment of one row, and the 4 rows give 4
// independent loads in flight per lane.  x_t is re-read by every row and
// stays in L1 / L2.
#include "pertime.cuh"

namespace wc4d {
namespace {

__global__ void __launch_bounds__(PT_THREADS) pertime_kernel(PtLayout L, PtProd op, const int* __restrict__ done,
                                                              int* ran) {
  pdl_wait();
  pdl_trigger();
  if (done != nullptr && *(volatile const int*)done) return;
  if (ran != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *ran = 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int task = blockIdx.x; task < L.tasks; task += gridDim.x) {
    // time level of this task: the last t with taskoff[t] <= task
    int lo = 0, hi = L.N1 - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (L.taskoff[mid] <= task) lo = mid;
      else hi = mid - 1;
    }
    const int t = lo;
    const int p = L.pt[t];
    const int r0 = (task - L.taskoff[t]) * PT_ROWS + warp * (PT_ROWS / 8);
    const double* A = op.A + L.aoff[t];
    const double* x = op.X + L.nuoff[t];
    constexpr int RW = PT_ROWS / 8;  // rows per warp
    double acc[RW];
#pragma unroll
    for (int q = 0; q < RW; ++q) acc[q] = 0.0;
    // k range covering every row of this warp (the triangle is masked per row)
    int k0 = 0, k1 = p;
    if (op.tri == TRI_LOWER) k1 = min(p, r0 + RW);
    if (op.tri == TRI_UPPER) k0 = min(p, r0) & ~31;
    for (int k = k0 + lane; k < k1; k += 32) {
      const double xk = x[k];
#pragma unroll
      for (int q = 0; q < RW; ++q) {
        const int i = r0 + q;
        const bool in = i < p && (op.tri == TRI_FULL || (op.tri == TRI_LOWER ? k <= i : k >= i));
        if (in) acc[q] = fma(A[(int64_t)i * p + k], xk, acc[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < RW; ++q) {
      double v = acc[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      const int i = r0 + q;
      if (lane == 0 && i < p) {
        const int64_t e = L.nuoff[t] + i;
        double val = v;
        if (op.mode == EPI_SADDLE_C2) val += op.v3[(int64_t)t * L.s + L.obs[e]];
        op.C[e] = val;
        if (op.Ch != nullptr) {
          const float h = (float)val;
          op.Ch[e] = h;
          op.Cl[e] = (float)(val - (double)h);
        }
      }
    }
  }
}

}  // namespace

void launch_pertime(const PtLayout& L, const PtProd& op, double bytes, const int* done, cudaStream_t st) {
  if (L.tasks <= 0) return;
  const int grid = std::min(L.tasks, 152 * 8);
  int* ran = prof_enabled() ? prof_begin(PROF_PERTIME, bytes, st) : nullptr;
  WC4D_CUDA(launch_pdl(pertime_kernel, dim3(grid), dim3(PT_THREADS), 0, st, L, op, done, ran));
  WC4D_LAUNCH_CHECK();
  if (ran) prof_end(st);
}

}  // namespace wc4d
