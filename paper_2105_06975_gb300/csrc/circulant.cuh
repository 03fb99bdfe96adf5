// Circulant covariance products by FFT (Sec. 6.1: on the periodic uniform
// grid the SOAR B and Q are circulant, so F B F^{-1} is diagonal).  Kernels
// in circulant.cu.
#pragma once
#include "common.cuh"

namespace wc4d {

constexpr int CIRC_P = 8;          // CTAs per cluster: one complex transform is split over 8 SMs
constexpr int CIRC_THREADS = 128;
constexpr int CIRC_MAX_JOBS = 4;
constexpr int CIRC_SMIN = 64;      // s = 8 Q with Q a power of two, 8 <= Q <= 1024
constexpr int CIRC_SMAX = 8192;

// s is a size the circulant kernels handle
inline bool circ_size_ok(int s) { return s >= CIRC_SMIN && s <= CIRC_SMAX && (s & (s - 1)) == 0; }

// One circulant product C = op(X) of ncols columns of length s with the
// spectrum lam (cluster layout, below), and the split-K reduction's epilogue
// (EPI_* of common.cuh) on each output column c (time t0 + c).
struct CircJob {
  const double* X;
  int64_t ldx;
  int ncols;
  const double* lam;  // FP64 kernel: spectrum in cluster layout
  int mode;
  double* C;
  int64_t ldc;
  int t0;
  const double* v3;  // EPI_SADDLE_C1: x part of the input vector
  const double* Y;   // EPI_SUB_FROM: minuend
  float* Ch = nullptr;  // optional double-float split of C
  float* Cl = nullptr;
  const float2* lamdf = nullptr;  // double-float kernel: the same spectrum as (hi, lo) pairs
};
struct CircJobs {
  CircJob j[CIRC_MAX_JOBS];
  int n = 0;
  int df = 0;  // 1: transforms in double-float on the FP32 pipe (DF32 / OZAKI modes), 0: FP64
  int tr_base[CIRC_MAX_JOBS + 1];  // complex transforms (column pairs) before each job
};

// flag = 1 unless the s x s matrix A equals the circulant of its first column
// to tol times its diagonal (setup of caller-given dense B, Q)
void launch_circ_check(const double* A, int s, double tol, int* flag, cudaStream_t st);
// Twiddle table tw[j] = exp(-2 pi i j / s), j < s (setup)
void launch_circ_twiddles(double2* tw, int s, cudaStream_t st);
// Spectrum of the symmetric circulant whose first column is col:
// lambda_k = sum_j col[j] cos(2 pi j k / s), accumulated in double-double.
// Written in the kernels' cluster layout, lam[(k mod 8) Q + bitrev_Q(k / 8)]
// = f(lambda_k) with f(x) = x + shift, or 1 / (x + shift) when invert != 0.
// flag (device int) is set to 1 if any lambda_k + shift is not positive and
// finite (the matrix is not SPD).
void launch_circ_spectrum(const double* col, int s, const double2* tw, double shift, int invert, double* lam,
                          int* flag, cudaStream_t st);
// all jobs of one launch (products of one dependency level); twdf: the
// twiddle table as double-float pairs (re, im), needed when jobs.df
void launch_circ(const CircJobs& jobs, int s, const double2* tw, const float4* twdf, const ModelDev& md,
                 const int* done, cudaStream_t st);
// out[i] = (hi, lo) of in[i] (setup: the double-float tables)
void launch_circ_split(const double* in, float2* out, int n, cudaStream_t st);
// add a job (transforms counted per pair of columns)
inline void circ_add(CircJobs& jobs, const CircJob& jb) {
  if (jobs.n == 0) jobs.tr_base[0] = 0;
  jobs.j[jobs.n] = jb;
  jobs.tr_base[jobs.n + 1] = jobs.tr_base[jobs.n] + (jb.ncols + 1) / 2;
  ++jobs.n;
}

// Banded circulant products (the modified SOAR B and Q of the heat-equation
// experiments, Sec. 6.1): y_j = delta x_j + sum_{|i| <= mv} row[i + mv]
// x_{(j + i) mod s}, 2 mv + 1 taps, symmetric (row[mv + i] = row[mv - i]).
// The epilogues of the circulant jobs apply (mode, C, ldc, t0, v3, Y, Ch, Cl).
struct BandJob {
  const double* X;
  int64_t ldx;
  int ncols;
  const double* row;  // device, 2 mv + 1 taps
  int mv;
  double delta;
  int mode;
  double* C;
  int64_t ldc;
  int t0;
  const double* v3;
  const double* Y;
  float* Ch = nullptr;
  float* Cl = nullptr;
};
struct BandJobs {
  BandJob j[CIRC_MAX_JOBS];
  int n = 0;
};
constexpr int BAND_TILE = 1024;  // outputs per CTA
void launch_band(const BandJobs& jobs, int s, const ModelDev& md, const int* done, cudaStream_t st);
// lambda_min of the symmetric banded circulant with taps row (setup): written
// to *out (device double) as the minimum over k of
// row[mv] + 2 sum_{i >= 1} row[mv + i] cos(2 pi i k / s)
void launch_band_lambda_min(const double* row, int mv, int s, double* out, cudaStream_t st);

}  // namespace wc4d
