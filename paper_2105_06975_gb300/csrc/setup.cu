// Setup kernels: SOAR covariances (Sec. 6.1), FP64 Cholesky of Dhat / Rhat,
// inverse triangular factors, the cyclic Jacobi eigensolver behind Alg. 1/2,
// and small utilities.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace wc4d {

static inline int nblk(int64_t n, int t = 256) { return (int)std::min<int64_t>((n + t - 1) / t, 152 * 16); }

// ------------------------------------------------------------------ SOAR
// c(r) = sigma2 (1 + r/ell) exp(-r/ell), r = chordal distance on the circle of
// circumference 1 between x_i = idx_i/s and x_j = idx_j/s: sin(pi |dx|)/pi.
// Entries depend only on the grid distance d = |idx_i - idx_j| in [0, s): the
// s correlations are evaluated once into a table (the exponential and sine
// run on GB300's 1/64-rate FP64 pipe) and the matrix is filled by lookup.
__global__ void soar_table_kernel(double* tab, int s, double sigma2, double ell) {
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < s; d += gridDim.x * blockDim.x) {
    const double r = sin(M_PI * ((double)d / s)) / M_PI;
    const double q = r / ell;
    tab[d] = sigma2 * (1.0 + q) * exp(-q);
  }
}
__global__ void soar_fill_kernel(double* M, int m, const int* idx, const double* __restrict__ tab) {
  const int64_t total = (int64_t)m * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int i, j;
    idx_divmod(e, m, total < ((int64_t)1 << 31), j, i);
    const int a = idx ? idx[i] : i, b = idx ? idx[j] : j;
    M[e] = tab[a > b ? a - b : b - a];
  }
}
void launch_soar_fill(double* M, int m, const int* idx, int s, double sigma2, double ell, double* tab,
                      cudaStream_t st) {
  soar_table_kernel<<<nblk(s), 256, 0, st>>>(tab, s, sigma2, ell);
  WC4D_LAUNCH_CHECK();
  soar_fill_kernel<<<nblk((int64_t)m * m), 256, 0, st>>>(M, m, idx, tab);
  WC4D_LAUNCH_CHECK();
}

// --------------------------------------------------------------- utilities
__global__ void copy_kernel(double* d, const double* s, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) d[e] = s[e];
}
void launch_copy_d(double* dst, const double* src, int64_t n, cudaStream_t st) {
  if (n > 0) copy_kernel<<<nblk(n), 256, 0, st>>>(dst, src, n);
  WC4D_LAUNCH_CHECK();
}
__global__ void fill_kernel(double* d, double v, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) d[e] = v;
}
void launch_fill_d(double* dst, double v, int64_t n, cudaStream_t st) {
  if (n > 0) fill_kernel<<<nblk(n), 256, 0, st>>>(dst, v, n);
  WC4D_LAUNCH_CHECK();
}
__global__ void add_diag_kernel(double* A, int m, int64_t lda, const double* sd, double sh) {
  const double v = sd ? *sd : sh;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) A[i + i * lda] += v;
}
void launch_add_diag(double* A, int m, int64_t lda, const double* shift_dev, double shift, cudaStream_t st) {
  add_diag_kernel<<<nblk(m), 256, 0, st>>>(A, m, lda, shift_dev, shift);
  WC4D_LAUNCH_CHECK();
}
__global__ void keep_diag_kernel(double* A, int m) {
  const int64_t total = (int64_t)m * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    if (e % m != e / m) A[e] = 0.0;
}
void launch_keep_diag(double* A, int m, cudaStream_t st) {
  keep_diag_kernel<<<nblk((int64_t)m * m), 256, 0, st>>>(A, m);
  WC4D_LAUNCH_CHECK();
}

// Alg. 3: sum of squares of the first super-diagonal block (rows pst[j] ..
// pst[j+1]-1, columns pst[j+1] .. pst[j+2]-1) of the m x m matrix A, one CTA
// per block j < nblocks
__global__ void __launch_bounds__(256) block_sumsq_kernel(const double* __restrict__ A, int m,
                                                          const int* __restrict__ pst, double* __restrict__ out) {
  __shared__ double red[8];
  const int j = blockIdx.x;
  const int r0 = pst[j], r1 = pst[j + 1], c1 = pst[j + 2];
  const int rows = r1 - r0;
  const int64_t cnt = (int64_t)rows * (c1 - r1);
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int r = r0 + (int)(e % rows), c = r1 + (int)(e / rows);
    const double a = A[r + (int64_t)c * m];
    acc = fma(a, a, acc);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[j] = t;
  }
}
void launch_block_sumsq(const double* A, int m, const int* pst, int nblocks, double* out, cudaStream_t st) {
  if (nblocks <= 0) return;
  block_sumsq_kernel<<<nblocks, 256, 0, st>>>(A, m, pst, out);
  WC4D_LAUNCH_CHECK();
}

// A[i + j m] = 0 where rows i and j lie in different runs (run[i] != run[j])
__global__ void zero_across_runs_kernel(double* A, int m, const int* __restrict__ run) {
  const int64_t total = (int64_t)m * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    if (run[e % m] != run[e / m]) A[e] = 0.0;
}
void launch_zero_across_runs(double* A, int m, const int* run, cudaStream_t st) {
  zero_across_runs_kernel<<<nblk((int64_t)m * m), 256, 0, st>>>(A, m, run);
  WC4D_LAUNCH_CHECK();
}
// At[j + i m] = A[i + j m], 32x32 tiles through shared memory
__global__ void transpose_kernel(const double* A, double* At, int m) {
  __shared__ double tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int i = bx + threadIdx.x, j = by + k;
    if (i < m && j < m) tile[k][threadIdx.x] = A[i + (int64_t)j * m];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int j = by + threadIdx.x, i = bx + k;
    if (i < m && j < m) At[j + (int64_t)i * m] = tile[threadIdx.x][k];
  }
}
void launch_transpose(const double* A, double* At, int m, cudaStream_t st) {
  dim3 g((m + 31) / 32, (m + 31) / 32), b(32, 8);
  transpose_kernel<<<g, b, 0, st>>>(A, At, m);
  WC4D_LAUNCH_CHECK();
}
__global__ void symmetrize_kernel(double* A, int m) {
  const int64_t total = (int64_t)m * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    if (i > j) {
      const double v = 0.5 * (A[e] + A[j + (int64_t)i * m]);
      A[e] = v;
      A[j + (int64_t)i * m] = v;
    }
  }
}
void launch_symmetrize(double* A, int m, cudaStream_t st) {
  symmetrize_kernel<<<nblk((int64_t)m * m), 256, 0, st>>>(A, m);
  WC4D_LAUNCH_CHECK();
}
__global__ void to_float_kernel(const double* a, float* b, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    b[e] = (float)a[e];
}
void launch_to_float(const double* a, float* b, int64_t n, cudaStream_t st) {
  if (n > 0) to_float_kernel<<<nblk(n), 256, 0, st>>>(a, b, n);
  WC4D_LAUNCH_CHECK();
}
__global__ void split_df_kernel(const double* a, float* hi, float* lo, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = a[e];
    const float h = __double2float_rn(v);
    hi[e] = h;
    lo[e] = __double2float_rn(v - (double)h);
  }
}
void launch_split_df(const double* a, float* hi, float* lo, int64_t n, cudaStream_t st) {
  if (n > 0) split_df_kernel<<<nblk(n), 256, 0, st>>>(a, hi, lo, n);
  WC4D_LAUNCH_CHECK();
}
// 32-bit index arithmetic (m * ncols < 2^31 is checked by the launcher): a
// 64-bit division per element is a long emulated sequence on the GPU
__global__ void split_df_block_kernel(const double* a, int64_t ld, int m, int ncols, float* hi, float* lo) {
  const int total = m * ncols;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int i = e % m, c = e / m;
    const double v = a[i + (int64_t)c * ld];
    const float h = __double2float_rn(v);
    hi[e] = h;
    lo[e] = __double2float_rn(v - (double)h);
  }
}
void launch_split_df_block(const double* a, int64_t ld, int m, int ncols, float* hi, float* lo, cudaStream_t st) {
  const int64_t n = (int64_t)m * ncols;
  WC4D_CHECK(n < ((int64_t)1 << 31), WC4D_ERR_ARG, "operand block too large for the split kernel");
  if (n > 0) split_df_block_kernel<<<nblk(n), 256, 0, st>>>(a, ld, m, ncols, hi, lo);
  WC4D_LAUNCH_CHECK();
}
// All operand blocks of one product launch split in one kernel: block o is
// an m_o x ncols_o column-major slice (leading dimension ld_o) written densely
// from offset off_o of hi / lo.
__global__ void split_df_multi_kernel(SplitBlocks sb, float* hi, float* lo) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < sb.total; g += gridDim.x * blockDim.x) {
    int o = 0;
    while (o + 1 < sb.n && g >= sb.off[o + 1]) ++o;
    const int e = g - sb.off[o];
    const int c = e / sb.m[o], i = e - c * sb.m[o];
    const double v = sb.a[o][i + (int64_t)c * sb.ld[o]];
    const float h = __double2float_rn(v);
    hi[g] = h;
    lo[g] = __double2float_rn(v - (double)h);
  }
}
void launch_split_df_multi(const SplitBlocks& sb, float* hi, float* lo, cudaStream_t st) {
  WC4D_CHECK(sb.total >= 0 && sb.total < (1 << 30), WC4D_ERR_ARG, "operand blocks too large for the split kernel");
  if (sb.total > 0) split_df_multi_kernel<<<nblk(sb.total), 256, 0, st>>>(sb, hi, lo);
  WC4D_LAUNCH_CHECK();
}

// inverse observation map: inv[j] = r if obs[r] == j, else -1
__global__ void inv_map_kernel(const int* obs, int p, int* inv, int s) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < p; r += gridDim.x * blockDim.x) inv[obs[r]] = r;
}
void launch_inv_map(const int* obs, int p, int* inv, int s, cudaStream_t st) {
  WC4D_CUDA(cudaMemsetAsync(inv, 0xff, sizeof(int) * s, st));
  inv_map_kernel<<<nblk(p), 256, 0, st>>>(obs, p, inv, s);
  WC4D_LAUNCH_CHECK();
}
// flag = 1 unless 0 <= obs[0] < obs[1] < ... < obs[p-1] < s
__global__ void check_obs_kernel(const int* obs, int p, int s, int* flag) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < p; r += gridDim.x * blockDim.x) {
    const int v = obs[r];
    if (v < 0 || v >= s || (r > 0 && obs[r - 1] >= v)) atomicExch(flag, 1);
  }
}
void launch_check_obs(const int* obs, int p, int s, int* flag, cudaStream_t st) {
  check_obs_kernel<<<nblk(p), 256, 0, st>>>(obs, p, s, flag);
  WC4D_LAUNCH_CHECK();
}
__global__ void check_finite_kernel(const double* a, int64_t n, int* flag) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(a[e])) atomicExch(flag, 1);
}
void launch_check_finite(const double* a, int64_t n, int* flag, cudaStream_t st) {
  if (n > 0) check_finite_kernel<<<nblk(n), 256, 0, st>>>(a, n, flag);
  WC4D_LAUNCH_CHECK();
}

// --------------------------------------------------------------- tile products
// acc[i][j] += sum_l A(r,l) B(l,c) over a tile, with A(r,l) = a[(ar0+r) +
// (ac0+l)*lda] (column-major, rows contiguous) and B(l,c) either
// b[(br0+l) + (bc0+c)*ldb] (BT = false) or b[(br0+c) + (bc0+l)*ldb] (BT = true:
// B given through its transpose).  Rows >= rlim / cols >= clim read 0.
struct TileMat {
  const double* p;
  int64_t ld;
  int r0, c0;
  int rlim, clim;  // valid extent in the (row, col) of the stored matrix
};
// 32x32 tiles with 64 threads (thread (tx, ty) = (tid % 8, tid / 8) owns rows
// tx + 8i and columns ty + 8j, i, j < 4): four times the CTAs of the 64x64 form
// for the same product, so small trailing matrices still spread over all SMs
// (GB300's FP64 pipe makes one 64x64x64 tile about 60 us on one SM).
template <bool BT>
__device__ void tile_mm32(double acc[4][4], const TileMat& A, const TileMat& B, int K, double (*As)[33],
                          double (*Bs)[33]) {
  const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
  for (int l0 = 0; l0 < K; l0 += 16) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + 64 * q;
      const int r = e & 31, kk = e >> 5;
      const int gr = A.r0 + r, gc = A.c0 + l0 + kk;
      As[kk][r] = (l0 + kk < K && gr < A.rlim && gc < A.clim) ? A.p[gr + (int64_t)gc * A.ld] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + 64 * q;
      if (!BT) {
        const int kk = e & 15, c = e >> 4;
        const int gr = B.r0 + l0 + kk, gc = B.c0 + c;
        Bs[kk][c] = (l0 + kk < K && gr < B.rlim && gc < B.clim) ? B.p[gr + (int64_t)gc * B.ld] : 0.0;
      } else {
        const int c = e & 31, kk = e >> 5;
        const int gr = B.r0 + c, gc = B.c0 + l0 + kk;
        Bs[kk][c] = (l0 + kk < K && gr < B.rlim && gc < B.clim) ? B.p[gr + (int64_t)gc * B.ld] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 8 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 8 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
}

// --------------------------------------------------------------- Cholesky
constexpr int NB = 64;

// Factor the nb x nb diagonal block at (j0, j0) in shared memory (unblocked,
// right-looking).  A non-positive or non-finite pivot records its 1-based
// index in *info (first one wins) and continues with pivot 1.  Step c updates
// only the active triangle i >= j > c, walked densely through a packed
// (row, column) table so every FP64 instruction of the step has work (GB300's
// FP64 pipe charges a warp instruction whether or not its lanes are active).
constexpr int TRI63 = (NB - 1) * NB / 2;  // entries of a size-63 lower triangle
__global__ void __launch_bounds__(256) potrf_diag_kernel(double* A, int64_t lda, int j0, int nb, int* info) {
  __shared__ double S[NB][NB + 1];
  __shared__ unsigned short tri[TRI63];  // e -> (i' << 8) | j', rows i' in order, 0 <= j' <= i'
  const int tid = threadIdx.x;
  for (int e = tid; e < NB * NB; e += 256) {
    const int i = e % NB, j = e / NB;
    S[i][j] = (i < nb && j < nb && i >= j) ? A[(j0 + i) + (int64_t)(j0 + j) * lda] : 0.0;
  }
  for (int e = tid; e < TRI63; e += 256) {
    int r = (int)((sqrtf(8.f * e + 1.f) - 1.f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= e) ++r;
    while (r * (r + 1) / 2 > e) --r;
    tri[e] = (unsigned short)((r << 8) | (e - r * (r + 1) / 2));
  }
  __syncthreads();
  for (int c = 0; c < nb; ++c) {
    if (tid == 0) {
      double d = S[c][c];
      if (!(d > 0.0) || !isfinite(d)) {
        atomicCAS(info, 0, j0 + c + 1);
        d = 1.0;
      }
      S[c][c] = sqrt(d);
    }
    __syncthreads();
    const double piv = S[c][c];
    for (int i = c + 1 + tid; i < nb; i += 256) S[i][c] /= piv;
    __syncthreads();
    const int rem = nb - c - 1, cnt = rem * (rem + 1) / 2;
    for (int e = tid; e < cnt; e += 256) {
      const int ij = tri[e];
      const int i = c + 1 + (ij >> 8), j = c + 1 + (ij & 255);
      S[i][j] = fma(-S[i][c], S[j][c], S[i][j]);
    }
    __syncthreads();
  }
  for (int e = tid; e < nb * nb; e += 256) {
    const int i = e % nb, j = e / nb;
    A[(j0 + i) + (int64_t)(j0 + j) * lda] = (i >= j) ? S[i][j] : 0.0;
  }
}

// Panel: rows i >= j0+nb solve x L11^T = a.  One CTA per 32 rows (lane =
// row), eight warps: warp w owns columns 8w..8w+7.  For column block b, warp b
// finishes its eight columns by substitution and publishes them; warps w > b
// subtract their contribution.  Every x_c accumulates its terms in increasing
// l with the same FMAs and division as a one-thread-per-row substitution (the
// results are identical), but the FP64 work of a row spreads over the four
// SM sub-partitions instead of one lane's serial chain.
__global__ void __launch_bounds__(256) trsm_panel_kernel(double* A, int64_t lda, int m, int j0, int nb) {
  __shared__ double L11[NB][NB];  // 32 KB
  __shared__ double X[NB][32];    // solved x_c of the CTA's 32 rows (16 KB)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    const int i = e % NB, j = e / NB;
    L11[i][j] = (i < nb && j < nb) ? A[(j0 + i) + (int64_t)(j0 + j) * lda] : (i == j ? 1.0 : 0.0);
  }
  const int row = j0 + nb + blockIdx.x * 32 + lane;
  const bool valid = row < m;
  double a[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int c = 8 * warp + q;
    a[q] = (valid && c < nb) ? A[row + (int64_t)(j0 + c) * lda] : 0.0;
  }
  __syncthreads();
  for (int b = 0; b < NB / 8; ++b) {
    if (warp == b) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int c = 8 * b + q;
        double v = a[q];
#pragma unroll
        for (int l = 0; l < q; ++l) v -= X[8 * b + l][lane] * L11[c][8 * b + l];
        X[c][lane] = v / L11[c][c];
      }
    }
    __syncthreads();
    if (warp > b) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int c = 8 * warp + q;
#pragma unroll
        for (int l = 0; l < 8; ++l) a[q] -= X[8 * b + l][lane] * L11[c][8 * b + l];
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int c = 8 * warp + q;
    if (valid && c < nb) A[row + (int64_t)(j0 + c) * lda] = X[c][lane];
  }
}

// Trailing update A[i][j] -= sum_l L[i][j0+l] L[j][j0+l] on lower-triangle
// 32x32 tiles (64 threads each).
__global__ void __launch_bounds__(64) syrk_update_kernel(double* A, int64_t lda, int m, int j0, int nb) {
  const int bi = blockIdx.x, bj = blockIdx.y;
  if (bj > bi) return;
  __shared__ double As[16][33];
  __shared__ double Bs[16][33];
  const int start = j0 + nb;
  const int r0 = start + bi * 32, c0 = start + bj * 32;
  double acc[4][4] = {};
  TileMat Am{A, lda, r0, j0, m, j0 + nb};
  TileMat Bm{A, lda, c0, j0, m, j0 + nb};
  tile_mm32<true>(acc, Am, Bm, nb, As, Bs);
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = r0 + tx + 8 * i, c = c0 + ty + 8 * j;
      if (r < m && c < m && r >= c) A[r + (int64_t)c * lda] -= acc[i][j];
    }
}

__global__ void zero_upper_kernel(double* A, int m) {
  const int64_t total = (int64_t)m * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int c, r;
    idx_divmod(e, m, total < ((int64_t)1 << 31), c, r);
    if (r < c) A[e] = 0.0;
  }
}

void cholesky(double* A, int m, int* info, cudaStream_t st, double* /*scratch*/) {
  for (int j0 = 0; j0 < m; j0 += NB) {
    const int nb = std::min(NB, m - j0);
    potrf_diag_kernel<<<1, 256, 0, st>>>(A, m, j0, nb, info);
    WC4D_LAUNCH_CHECK();
    const int rem = m - j0 - nb;
    if (rem > 0) {
      trsm_panel_kernel<<<(rem + 31) / 32, 256, 0, st>>>(A, m, m, j0, nb);
      WC4D_LAUNCH_CHECK();
      const int T = (rem + 31) / 32;
      syrk_update_kernel<<<dim3(T, T), 64, 0, st>>>(A, m, m, j0, nb);
      WC4D_LAUNCH_CHECK();
    }
  }
  zero_upper_kernel<<<nblk((int64_t)m * m), 256, 0, st>>>(A, m);
  note_launch();
  WC4D_LAUNCH_CHECK();
}

// ------------------------------------------------------ triangular inverse
// Diagonal blocks: Dinv_b = (L_bb)^{-1}, stored as 64x64 column-major blocks.
__global__ void __launch_bounds__(64) trtri_diag_kernel(const double* L, int64_t lda, int m, double* Dinv) {
  __shared__ double S[NB][NB + 1];
  __shared__ double X[NB][NB + 1];
  const int b = blockIdx.x, j0 = b * NB;
  const int nb = min(NB, m - j0);
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int i = e % NB, j = e / NB;
    S[i][j] = (i < nb && j < nb) ? L[(j0 + i) + (int64_t)(j0 + j) * lda] : (i == j ? 1.0 : 0.0);
  }
  __syncthreads();
  const int c = threadIdx.x;  // column of the inverse
  for (int r = 0; r < NB; ++r) {
    double v = (r == c) ? 1.0 : 0.0;
    if (r >= c) {
      for (int l = c; l < r; ++l) v -= S[r][l] * X[l][c];
      v /= S[r][r];
    } else {
      v = 0.0;
    }
    X[r][c] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int i = e % NB, j = e / NB;
    Dinv[(int64_t)b * NB * NB + e] = X[i][j];
  }
}

// Blocked inverse W = L^{-1} (NB-row blocks, Dinv_i = L_ii^{-1}).  Forward
// substitution on the identity E: for each block row i in turn,
//   E[j, cb] -= (L_ji Dinv_i) E[i, cb]   for j > i, cb <= i,
// and at the end W[i, cb] = Dinv_i E[i, cb] for all i, cb <= i at once (the
// same products as scaling block row i before it is used, regrouped so that
// only the updates form a serial chain).  All products on 32x32 tiles.

// M_ji = L_ji Dinv_i for every block pair j > i (one launch; M in the layout of L)
__global__ void __launch_bounds__(64) trinv_scale_kernel(const double* L, double* M, int m, const double* Dinv) {
  const int nbk = (m + NB - 1) / NB;
  int pair = blockIdx.x >> 2;  // (j, i) with j > i, enumerated row by row: j = 1.., i = 0..j-1
  int j = 1;
  while (pair >= j) {
    pair -= j;
    ++j;
  }
  const int i = pair, sub = blockIdx.x & 3;
  if (j >= nbk) return;
  __shared__ double As[16][33];
  __shared__ double Bs[16][33];
  const int r0 = j * NB + 32 * (sub & 1), cs = 32 * (sub >> 1);
  double acc[4][4] = {};
  TileMat Am{L, m, r0, i * NB, m, m};
  TileMat Bm{Dinv + (int64_t)i * NB * NB, NB, 0, cs, NB, NB};
  tile_mm32<false>(acc, Am, Bm, NB, As, Bs);
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int r = r0 + tx + 8 * a, c = i * NB + cs + ty + 8 * b;
      if (r < m) M[r + (int64_t)c * m] = acc[a][b];
    }
}

// Step i: E[j, cb] -= M_ji E[i, cb] for block rows j > i, block columns cb <= i
// (reads block row i, writes the rows below it: no overlap).
__global__ void __launch_bounds__(64) trinv_update_kernel(const double* M, double* W, int m, int i) {
  const int nsub = 4 * (i + 1);  // 32x32 sub-tiles per block row
  const int jb = i + 1 + blockIdx.x / nsub, t = blockIdx.x % nsub;
  const int cb = t >> 2, sub = t & 3;
  __shared__ double As[16][33];
  __shared__ double Bs[16][33];
  const int r0 = jb * NB + 32 * (sub & 1), c0 = cb * NB + 32 * (sub >> 1), k0 = i * NB;
  double acc[4][4] = {};
  TileMat Am{M, m, r0, k0, m, m};
  TileMat Bm{W, m, k0, c0, m, m};
  tile_mm32<false>(acc, Am, Bm, NB, As, Bs);
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int r = r0 + tx + 8 * a, c = c0 + ty + 8 * b;
      if (r < m && c < m) W[r + (int64_t)c * m] -= acc[a][b];
    }
}

// W[i, cb] = Dinv_i E[i, cb] in place for every i and cb <= i: one CTA per
// (block row, 32-column stripe) reads its whole 64 x 32 input before writing.
__global__ void __launch_bounds__(128) trinv_finish_kernel(double* W, int m, const double* Dinv) {
  int t = blockIdx.x >> 1;  // (i, cb) with cb <= i, row by row
  int i = 0;
  while (t > i) {
    t -= i + 1;
    ++i;
  }
  const int cb = t, half = blockIdx.x & 1;
  const int r0 = i * NB, c0 = cb * NB + 32 * half;
  const int nb = min(NB, m - r0);
  __shared__ double Dt[NB][NB];  // Dt[k][r] = Dinv_i(r, k): lanes of a warp read consecutive r
  __shared__ double E[NB][32];   // E[i, stripe]  (48 KB together)
  const int tid = threadIdx.x;
  for (int e = tid; e < NB * NB; e += 128) Dt[e / NB][e % NB] = Dinv[(int64_t)i * NB * NB + e];
  for (int e = tid; e < NB * 32; e += 128) {
    const int r = e % NB, c = e / NB;
    E[r][c] = (r < nb && c0 + c < m) ? W[(r0 + r) + (int64_t)(c0 + c) * m] : 0.0;
  }
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;  // rows tx + 16 a, columns ty + 8 b
  double acc[4][4] = {};
  for (int k = 0; k < nb; ++k) {
    double d[4], e[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) d[a] = Dt[k][tx + 16 * a];
#pragma unroll
    for (int b = 0; b < 4; ++b) e[b] = E[k][ty + 8 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(d[a], e[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int r = tx + 16 * a, c = c0 + ty + 8 * b;
      if (r < nb && c < m) W[(r0 + r) + (int64_t)c * m] = acc[a][b];
    }
}

__global__ void identity_kernel(double* W, int m) {
  const int64_t total = (int64_t)m * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int c, r;
    idx_divmod(e, m, total < ((int64_t)1 << 31), c, r);
    W[e] = (r == c) ? 1.0 : 0.0;
  }
}

// W = L^{-1} (the scheme above); Wt = W^T.  Wt serves as the M_ji buffer
// until the final transpose overwrites it.
void tri_inverse(const double* L, double* W, double* Wt, int m, cudaStream_t st, double* scratch) {
  const int nbk = (m + NB - 1) / NB;
  identity_kernel<<<nblk((int64_t)m * m), 256, 0, st>>>(W, m);
  note_launch();
  trtri_diag_kernel<<<nbk, 64, 0, st>>>(L, m, m, scratch);
  WC4D_LAUNCH_CHECK();
  if (nbk > 1) {
    trinv_scale_kernel<<<4 * (nbk * (nbk - 1) / 2), 64, 0, st>>>(L, Wt, m, scratch);
    WC4D_LAUNCH_CHECK();
    for (int i = 0; i + 1 < nbk; ++i) {
      trinv_update_kernel<<<(nbk - i - 1) * 4 * (i + 1), 64, 0, st>>>(Wt, W, m, i);
      WC4D_LAUNCH_CHECK();
    }
  }
  trinv_finish_kernel<<<2 * (nbk * (nbk + 1) / 2), 128, 0, st>>>(W, m, scratch);
  WC4D_LAUNCH_CHECK();
  launch_transpose(W, Wt, m, st);
}

// ------------------------------------------------------------- Jacobi eigen
// Cyclic Jacobi with the round-robin pairing: in round r (0..m-2) the pairs
// are (0, 1 + r mod (m-1)) and (1 + (r+i) mod (m-1), 1 + (r-i) mod (m-1)) for
// i = 1..m/2-1, so every pair meets once per sweep and the pairs of a round
// are disjoint.  A <- J^T A J, V <- V J with the 2x2 rotation
// [[c, s], [-s, c]], theta = atan2(2 a_pq, a_qq - a_pp) / 2, which zeroes a_pq.
__device__ __forceinline__ void rr_pair(int m, int r, int i, int& p, int& q) {
  const int n1 = m - 1;
  if (i == 0) {
    p = 0;
    q = 1 + r % n1;
  } else {
    p = 1 + (r + i) % n1;
    q = 1 + ((r - i) % n1 + n1) % n1;
  }
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
}

__global__ void jacobi_rot_kernel(const double* A, int m, int r, double* rot, int* count) {
  const int half = m / 2;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < half; i += gridDim.x * blockDim.x) {
    int p, q;
    rr_pair(m, r, i, p, q);
    const double app = A[p + (int64_t)p * m], aqq = A[q + (int64_t)q * m], apq = A[p + (int64_t)q * m];
    double c = 1.0, s = 0.0;
    if (fabs(apq) > 1e-300 && fabs(apq) > 1e-15 * sqrt(fabs(app * aqq))) {
      const double th = 0.5 * atan2(2.0 * apq, aqq - app);
      c = cos(th);
      s = sin(th);
      atomicAdd(count, 1);
    }
    rot[4 * i + 0] = p;
    rot[4 * i + 1] = q;
    rot[4 * i + 2] = c;
    rot[4 * i + 3] = s;
  }
}

// thread per 2x2 block (pair P1 rows, pair P2 columns) and per (row, pair) of V
__global__ void jacobi_apply_kernel(double* A, double* V, int m, const double* rot) {
  const int half = m / 2;
  const int64_t nA = (int64_t)half * half;
  const int64_t nV = (int64_t)m * half;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nA + nV; e += (int64_t)gridDim.x * blockDim.x) {
    if (e < nA) {
      const int i1 = (int)(e % half), i2 = (int)(e / half);
      const int p1 = (int)rot[4 * i1], q1 = (int)rot[4 * i1 + 1];
      const double c1 = rot[4 * i1 + 2], s1 = rot[4 * i1 + 3];
      const int p2 = (int)rot[4 * i2], q2 = (int)rot[4 * i2 + 1];
      const double c2 = rot[4 * i2 + 2], s2 = rot[4 * i2 + 3];
      if (s1 == 0.0 && s2 == 0.0) continue;
      double* a_pp = A + p1 + (int64_t)p2 * m;
      double* a_pq = A + p1 + (int64_t)q2 * m;
      double* a_qp = A + q1 + (int64_t)p2 * m;
      double* a_qq = A + q1 + (int64_t)q2 * m;
      const double m00 = *a_pp, m01 = *a_pq, m10 = *a_qp, m11 = *a_qq;
      // M J2 (columns)
      const double n00 = c2 * m00 - s2 * m01, n01 = s2 * m00 + c2 * m01;
      const double n10 = c2 * m10 - s2 * m11, n11 = s2 * m10 + c2 * m11;
      // J1^T (M J2) (rows)
      double o00 = c1 * n00 - s1 * n10, o01 = c1 * n01 - s1 * n11;
      double o10 = s1 * n00 + c1 * n10, o11 = s1 * n01 + c1 * n11;
      if (i1 == i2) {
        o01 = 0.0;
        o10 = 0.0;
      }
      *a_pp = o00;
      *a_pq = o01;
      *a_qp = o10;
      *a_qq = o11;
    } else {
      const int64_t f = e - nA;
      const int row = (int)(f % m), i2 = (int)(f / m);
      const double c = rot[4 * i2 + 2], s = rot[4 * i2 + 3];
      if (s == 0.0) continue;
      const int p = (int)rot[4 * i2], q = (int)rot[4 * i2 + 1];
      const double vp = V[row + (int64_t)p * m], vq = V[row + (int64_t)q * m];
      V[row + (int64_t)p * m] = c * vp - s * vq;
      V[row + (int64_t)q * m] = s * vp + c * vq;
    }
  }
}

int jacobi_eigh(double* A, double* V, int m, cudaStream_t st, double* rot, int* d_count, int max_sweeps) {
  identity_kernel<<<nblk((int64_t)m * m), 256, 0, st>>>(V, m);
  WC4D_LAUNCH_CHECK();
  if (m < 2) return 0;
  const int half = m / 2;
  const int64_t work = (int64_t)half * half + (int64_t)m * half;
  int sweeps = 0;
  for (; sweeps < max_sweeps; ++sweeps) {
    WC4D_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int), st));
    for (int r = 0; r < m - 1; ++r) {
      jacobi_rot_kernel<<<nblk(half), 256, 0, st>>>(A, m, r, rot, d_count);
      note_launch();
      jacobi_apply_kernel<<<nblk(work), 256, 0, st>>>(A, V, m, rot);
      note_launch();
    }
    WC4D_LAUNCH_CHECK();
    int h = 0;
    WC4D_CUDA(cudaMemcpyAsync(&h, d_count, sizeof(int), cudaMemcpyDeviceToHost, st));
    WC4D_CUDA(cudaStreamSynchronize(st));
    if (h == 0) {
      ++sweeps;
      break;
    }
  }
  return sweeps;
}

// U[k + i m] = sqrt(max(lambda_k, T)) * V[i + k m]  (U = Lambda_ME^{1/2} V^T), lambda_k = A[k][k]
__global__ void me_scale_kernel(const double* Ajac, const double* V, int m, double T, double* U) {
  const int64_t total = (int64_t)m * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % m), i = (int)(e / m);
    const double lam = Ajac[k + (int64_t)k * m];
    U[e] = sqrt(lam > T ? lam : T) * V[i + (int64_t)k * m];
  }
}
void launch_me_scale(const double* Ajac, const double* V, int m, double T, double* U, double*, cudaStream_t st) {
  me_scale_kernel<<<nblk((int64_t)m * m), 256, 0, st>>>(Ajac, V, m, T, U);
  WC4D_LAUNCH_CHECK();
}

}  // namespace wc4d
