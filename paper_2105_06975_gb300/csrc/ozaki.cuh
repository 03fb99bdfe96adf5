// Ozaki-scheme products on the tensor cores: digit forms and the tcgen05
// stream-K kernel (ozaki.cu).
#pragma once
#include "common.cuh"

namespace wc4d {

constexpr int OZ_DIGITS = 7;                 // balanced base-128 digits per operand (47 bits)
constexpr int OZ_BM = 128;                   // operator rows per tile (MMA M, TMEM lanes)
constexpr int OZ_BN = 64;                    // X columns per tile (MMA N)
constexpr int OZ_BK = 16;                    // k per MMA and per digit tile
constexpr int OZ_KMAX = 512;                 // longest k-range accumulated exactly in FP32
constexpr int OZ_GEMV_K = 128;               // longest k-range of a one-column (GEMV) segment
constexpr int OZ_A_TILE = OZ_BM * OZ_BK;     // elements of one operator digit tile
constexpr int OZ_X_TILE = OZ_BN * OZ_BK;     // elements of one X digit tile

// Digit form of the X operand of one op of a launch, and the double-float
// split of its one-column (GEMV) column if it has one.
struct OzColJob {
  const double* X;
  int64_t ldx;
  int kdim, ncols, nkb;
  uint16_t* Xd;  // oz_x_elems(kdim, ncols) BF16 digits
  float* Xs;     // oz_wide_tiles(ncols) * OZ_BN scales
  int wide;      // oz_wide_tiles(ncols)
  int gemv_col;  // oz_gemv_col(ncols), -1 if none
  float* Xgh;    // kdim floats each: hi / lo parts of column gemv_col
  float* Xgl;
};
struct OzColJobs {
  OzColJob j[GEMM_MAX_OPS];
  int cta_base[GEMM_MAX_OPS + 1];  // wide * 64 CTAs per op, + oz_gemv_ctas(kdim) with a GEMV column
  int n;
};

// the column a plan runs as a one-column (GEMV) tile: column 0 of a
// one-column op, the last column when ncols = 64 q + 1 (q >= 1); else -1
inline int oz_gemv_col(int ncols) {
  if (ncols == 1) return 0;
  if (ncols > OZ_BN && ncols % OZ_BN == 1) return ncols - 1;
  return -1;
}

// CTAs of the digit kernel that split an op's GEMV column (128 entries each)
inline int oz_gemv_ctas(int kdim) { return (kdim + 127) / 128; }
// column tiles of an op that run on the tensor cores (width >= 2)
int oz_wide_tiles(int ncols);
// BF16 elements of an operator's digit tiles (rows padded to 128, k to 16)
int64_t oz_operator_elems(int m, int kdim);
// BF16 elements of an X operand's digit tiles
int64_t oz_x_elems(int kdim, int ncols);
// operator digits (setup): rows i of op(At) (At[k + i lda], k < kdim);
// As gets ceil(m/128)*128 scales
void launch_oz_rows(const double* At, int64_t lda, int m, int kdim, uint16_t* Ad, float* As, cudaStream_t st);
// X digits of every op of one launch
void launch_oz_cols(const OzColJobs& jobs, cudaStream_t st);
// One-column products of a symmetric Toeplitz operator (every entry a function
// of |i - k|, as the SOAR covariances of the periodic uniform grid): the GEMV
// segments read the operator's split first row instead of its m x m entries,
// the same values in the same order (GemmOpT::Th).  Layout of the row copies:
inline int oz_toeplitz_off(int m) { return (m + 3) / 4 * 4; }
inline int64_t oz_toeplitz_stride(int m) { return 2 * (int64_t)oz_toeplitz_off(m) + 4; }
// setup: *flag (device) is set to 1 unless every entry At[i lda + k] of the
// m x m operator is bitwise equal to At[|i - k|]; Th / Tl (4 oz_toeplitz_stride(m)
// floats each) receive the copies of the first row of the split (Ah, Al),
// to be used only if the flag stays 0
void launch_oz_toeplitz(const double* At, int64_t lda, int m, const float* Ah, const float* Al, float* Th,
                        float* Tl, int* flag, cudaStream_t st);
// setup: *flag (device) is set to 1 unless every digit tile (R, K) of the
// operator's digit form (launch_oz_rows of an m x kdim operator) is bitwise
// equal to the tile of the same offset 128 R - 16 K that the product kernel
// then reads in its place (GemmOpT::toep_tiles)
void launch_oz_toeplitz_tiles(const uint16_t* Ad, int m, int kdim, int* flag, cudaStream_t st);
// the tensor-core stream-K products of a plan built with COST_TC; err (device
// int, may be NULL) receives a non-zero code if a wait gave up
void launch_gemm_tc(const GemmOpsT<double>& ops, const GemmSeg* segs, const int* seg_start, int nctas,
                    double* partial, const int* done, int* ran, int* err, cudaStream_t st);
// persistent CTAs of the tensor-core kernel (one per SM)
int oz_resident_ctas();
// process-wide time limit of the kernel's pipeline waits in ns (0: the default
// of 1 s); the final drain waits always keep the default
void oz_set_wait_limit(unsigned long long ns);
unsigned long long oz_wait_limit();

}  // namespace wc4d
