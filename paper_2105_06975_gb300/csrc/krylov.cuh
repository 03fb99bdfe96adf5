// Device-resident Krylov kernels (FP64 recurrences, deterministic reductions).
#pragma once
#include "common.cuh"

namespace wc4d {

constexpr int DOT_BLOCKS = 304;  // 2 per SM on a 152-SM GB300; fixed for deterministic sums
constexpr int DOT_THREADS = 256;
// block-dot partials of the Arnoldi passes: one partial per 1024-element chunk
constexpr int ORTH_U = 4;                         // elements per thread
constexpr int ORTH_G = 4;                         // basis vectors per block
constexpr int ORTH_CHUNK = DOT_THREADS * ORTH_U;  // elements per block
inline int orth_chunks(int64_t n) { return (int)((n + ORTH_CHUNK - 1) / ORTH_CHUNK); }
// Chunk count of the split-basis dot kernels for cnt basis vectors: at most
// three CTAs (chunks x vector groups) per SM, all resident at 80 registers
// (rounded down: a few CTAs beyond one wave would run as a second wave and
// nearly double the pass), so each thread strides over several float4 and the
// closing block reduction (a shuffle tree per vector) is amortised.  The
// partial buffer holds orth_chunks(n) >= this many partials per row.
inline int dot_chunks(int64_t n, int cnt) {
  const int maxc = orth_chunks(n);
  const int groups = (cnt + ORTH_G - 1) / ORTH_G;
  int c = (152 * 3) / groups;
  return c < 1 ? 1 : (c > maxc ? maxc : c);
}

// Chunk count of the delayed-CGS2 dot pass (DF32 / OZAKI GMRES): as
// dot_chunks, but two CTAs per SM, the residency its shared-memory copy ring
// (96 KB per CTA) allows.
inline int dc_dot_chunks(int64_t n, int cnt) {
  const int maxc = orth_chunks(n);
  const int groups = (cnt + ORTH_G - 1) / ORTH_G;
  int c = (152 * 2) / groups;
  return c < 1 ? 1 : (c > maxc ? maxc : c);
}

struct DevStatus {
  int done;
  int status;
  int iters;
  int pad;
  double est;      // recurrence residual estimate (relative)
  double tol_est;  // threshold the estimate is compared with
};

// MINRES scalar state (double buffered: read sc_in, block 0 writes sc_out)
enum { MS_GAMMA = 0, MS_GAMMA_OLD, MS_ETA, MS_ETA0, MS_C, MS_C_OLD, MS_S, MS_S_OLD, MS_COUNT };

template <typename T>
void dot_partial(const T* a, const T* b, int64_t n, double* part, const int* done, cudaStream_t st);
void dot_finish(const double* part, double* out, int sqrt_it, cudaStream_t st);

void minres_init(const double* part_gamma, double* sc, DevStatus* stat, double tol, cudaStream_t st);
void minres_v_update(const double* part_delta, const double* sc, const double* Az, const double* v,
                     const double* v_old, double* v_new, int64_t n, const int* done, cudaStream_t st);
void minres_update(const double* part_delta, const double* part_gamma, const double* sc_in, double* sc_out,
                   const double* z, const double* w_old, const double* w, double* w_new, double* x, int64_t n,
                   DevStatus* stat, cudaStream_t st);

// GMRES / FGMRES (Arnoldi with classical Gram-Schmidt and one reorthogonalisation)
template <typename T>
void gm_mdot(const T* V, int64_t ldv, int cnt, const T* w, int64_t n, double* part, const int* done,
             cudaStream_t st);
void gm_mdot_reduce(const double* part, int cnt, int nchunks, double* h, const int* done, cudaStream_t st);
template <typename T>
void gm_mupdate(const T* V, int64_t ldv, int cnt, const double* h, T* w, int64_t n, const int* done,
                cudaStream_t st);
template <typename T>
void gm_init(const T* r0, const double* part_beta, T* v0, double* g, DevStatus* stat, double tol, int64_t n,
             cudaStream_t st);
void gm_hessenberg(int j, const double* h1, const double* h2, const double* part_norm, double* H, int ldh,
                   double* cs, double* sn, double* g, double* hnext, DevStatus* stat, const double* bnorm,
                   cudaStream_t st);
template <typename T>
void gm_normalize(const T* w, const double* hnext, T* v, int64_t n, const int* done, cudaStream_t st);
void gm_solve_y(const double* H, int ldh, const double* g, int k, double* y, cudaStream_t st);
// as gm_solve_y with k = min(stat->iters, kmax) read on the device
void gm_solve_y_dev(const double* H, int ldh, const double* g, const DevStatus* stat, int kmax, double* y,
                    cudaStream_t st);
// x = sum_{i < min(stat->iters, kmax)} y_i Z_i  (FP64 accumulation)
template <typename T, typename TZ>
void gm_combine_dev(const TZ* Z, int64_t ldz, const DevStatus* stat, int kmax, const double* y, T* x, int64_t n,
                    cudaStream_t st);
template <typename T, typename TZ>
void gm_combine(const TZ* Z, int64_t ldz, int k, const double* y, const T* x0, T* x, int64_t n, cudaStream_t st);

// double-float Arnoldi basis (DF32 mode): basis vectors stored as FP32 hi/lo
// pairs; dots and updates run on the FP32 pipe with exact-error accumulation
void gm_mdot_df(const float* Vh, const float* Vl, int64_t ldv, int cnt, const float* wh, const float* wl, int64_t n,
                double* part, const int* done, cudaStream_t st);
void gm_mupdate_df(const float* Vh, const float* Vl, int64_t ldv, int cnt, const double* h, double* w, float* wh,
                   float* wl, int64_t n, const int* done, cudaStream_t st);
// v = w / hnext as a double vector and as its split into the basis slot
void gm_normalize_df(const double* w, const double* hnext, double* v, float* vh, float* vl, int64_t n,
                     const int* done, cudaStream_t st);
void gm_split(const double* w, float* wh, float* wl, int64_t n, const int* done, cudaStream_t st);
// the first vector of the delayed-CGS2 basis in its storage form: FP32 low
// parts, or BF16 low parts (16-bit words, same leading dimension) with b6
void gm_split_basis(const double* w, float* vh, float* vl, int64_t n, bool b6, cudaStream_t st);

// delayed CGS2 Arnoldi on the split basis (DF32 GMRES): scalar state slots
enum { DC_GAMMA = 0, DC_ALPHA, DC_IGAMMA, DC_IALPHA, DC_BETA, DC_COUNT };
// b6: the basis low parts are BF16 (6-byte entries), else FP32
// part: dot_chunks(n, j + 1) double-float partials per row (rows a_0..a_j | c_0..c_j | w^T w), summed by
// gm_dc_coef
void gm_dc_dot(const float* Vh, const float* Vl, int64_t ldv, int j, const float* wh, const float* wl, int64_t n,
               float2* part, const int* done, cudaStream_t st, bool b6);
// hc: Hbar c of the previous step (j rows), written by gm_dc_update
void gm_dc_coef(int j, const float2* part, int nchunks, double* dc, double* bprev, double* cprev, double* e,
                double* Hraw, double* H, double* T, int ldh, double* cs, double* sn, double* g, double* hnext,
                DevStatus* stat, const double* bnorm, const double* hc, cudaStream_t st);
void gm_dc_update(float* Vh, float* Vl, int64_t ldv, int j, const double* e, const double* c, const double* dc,
                  const double* w, double* v, int64_t n, const double* Hraw, int ldh, double* hc, const int* done,
                  cudaStream_t st, bool b6);

// small vector ops
template <typename T>
void vec_axpby(T* y, const T* x, double a, double b, int64_t n, cudaStream_t st);  // y = a x + b y
void vec_sub(const double* a, const double* b, double* out, int64_t n, cudaStream_t st);
template <typename TD, typename TS>
void vec_convert(const TS* src, TD* dst, int64_t n, double scale, cudaStream_t st);

}  // namespace wc4d
