// Per-time observation sets H_i and covariances R_i (Sec. 2.1: H and R are
// block diagonal over the time levels, each R_i of its own size p_i).  The R
// family of products becomes N+1 independent matrix-vector products, one per
// time level, run by one batched kernel (pertime.cu).
#pragma once
#include "common.cuh"

namespace wc4d {

// One batched product out_t = op(A_t) x_t for t = 0..N: A_t is the p_t x p_t
// block at A + aoff[t] (column-major, "TN" form op(A)_i = sum_k A[k + i p_t] x_k,
// k over the full range, k <= i (TRI_LOWER) or k >= i (TRI_UPPER)).  x and the
// output are nu-layout vectors: time t's entries start at nuoff[t].  Epilogue
// EPI_STORE or EPI_SADDLE_C2 (out = acc + v3_t[obs[nuoff[t] + r]]); optional
// double-float split of the output.  FP64 products in every precision mode
// (each operator entry is read once for one multiply-add).
struct PtProd {
  const double* A;
  int tri;
  const double* X;
  int mode;
  double* C;
  const double* v3 = nullptr;
  float* Ch = nullptr;
  float* Cl = nullptr;
};
struct PtLayout {
  int N1;                 // N + 1 time levels
  int s;                  // grid size (v3 stride)
  const int* pt;          // device [N+1]: p_t
  const int* nuoff;       // device [N+2]: prefix sums of p_t
  const int64_t* aoff;    // device [N+1]: element offset of block t
  const int* taskoff;     // device [N+2]: prefix sums of ceil(p_t / PT_ROWS)
  const int* obs;         // device [sum p_t]: the sets, one after another
  int tasks;              // taskoff[N+1]
};
constexpr int PT_ROWS = 32;     // rows per CTA task (4 per warp)
constexpr int PT_THREADS = 256;

// bytes: the launch's algorithmic bytes, recorded when profiling is on
void launch_pertime(const PtLayout& L, const PtProd& op, double bytes, const int* done, cudaStream_t st);

}  // namespace wc4d
