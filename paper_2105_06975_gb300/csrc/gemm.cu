// Stream-K batched GEMM for the multi-right-hand-side covariance products.
//
// Every covariance product of the method is C = Sigma * V with V the s x (N+1)
// (or p x (N+1)) time-block matrix of a Krylov vector: the D pass and R pass of
// A v (Sec. 6.2), the Dhat^{-1} / Rhat^{-1} solves (applied as products with
// the inverse Cholesky factors) and the D pass inside Shat^{-1} and P_I^{-1}.
// Several independent products of one dependency level go into one launch.
// The work (tiles x k-blocks, weighted by their multiply-adds) is cut into
// exactly equal contiguous ranges, one per persistent CTA, so every SM gets the
// same share of FP64 work; partial tiles are summed in a fixed order by the
// reduction, which also applies the fused epilogue (the L v3 / H v3 terms of
// A v, the v1 - D c1 of P_I).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <string>

#include "common.cuh"
#include "model_dev.cuh"
#include "ozaki.cuh"

namespace wc4d {

// --------------------------------------------------------------- planning
// A plan is a pure function of (device, op shapes, CTA count, cost model) and
// read-only on the device once built, so built plans are kept in a bounded
// process-wide cache and shared: a problem of the same shapes as an earlier
// one (the next assimilation window, a benchmark step) reuses its schedule
// instead of rebuilding it and paying for device allocations and copies.
namespace {
struct PlanArrays {
  void* p[4] = {nullptr, nullptr, nullptr, nullptr};
  ~PlanArrays() {
    for (void* q : p) cudaFree(q);
  }
};
std::mutex g_plan_mu;
std::map<std::string, GemmPlan>& plan_cache() {
  static std::map<std::string, GemmPlan> c;
  return c;
}
constexpr size_t PLAN_CACHE_MAX = 512;
}  // namespace

void plan_free(GemmPlan& plan) { plan = GemmPlan(); }

void plan_build(GemmPlan& plan, const std::vector<OpShape>& shapes, int max_ctas, int cost_model) {
  plan_free(plan);
  WC4D_CHECK((int)shapes.size() <= GEMM_MAX_OPS, WC4D_ERR_ARG, "too many GEMM ops in one launch");
  int dev = 0;
  WC4D_CUDA(cudaGetDevice(&dev));
  std::string key = std::to_string(dev) + ":" + std::to_string(max_ctas) + ":" + std::to_string(cost_model);
  for (const OpShape& sh : shapes)
    key += ":" + std::to_string(sh.m) + "," + std::to_string(sh.kdim) + "," + std::to_string(sh.ncols) + "," +
           std::to_string(sh.tri);
  {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto it = plan_cache().find(key);
    if (it != plan_cache().end()) {
      plan = it->second;
      return;
    }
  }
  plan.nops = (int)shapes.size();
  // the tensor-core plan: 128-row tiles, segments of at most OZ_KMAX k (exact
  // FP32 accumulation of the digit products)
  const bool tc = (cost_model == COST_TC);
  const int bm = tc ? OZ_BM : GEMM_BM;
  plan.bm = bm;
  struct Tile {
    int op, row0, col0, kb0, kb1;
    double cost_per_kb;
    bool gemv;
  };
  std::vector<Tile> tiles;
  int64_t outpos = 0;
  double flops = 0;
  for (int o = 0; o < plan.nops; ++o) {
    const OpShape& sh = shapes[o];
    WC4D_CHECK((int64_t)sh.m * sh.ncols < ((int64_t)1 << 31), WC4D_ERR_ARG, "GEMM output too large (2^31 entries)");
    plan.shape[o] = sh;
    const int rt = (sh.m + bm - 1) / bm;
    const int ct = std::max(1, (sh.ncols + GEMM_BN - 1) / GEMM_BN);
    // full 64-column tiles plus a remainder tile; a one-column remainder (the
    // 65th time level) runs on the GEMV mapping
    const int cw = std::min(GEMM_BN, std::max(1, sh.ncols));
    plan.tile_base[o] = (int)tiles.size();
    plan.col_tiles[o] = ct;
    plan.col_width[o] = cw;
    plan.out_base[o] = outpos;
    outpos += (int64_t)sh.m * sh.ncols;
    if (sh.m <= 0 || sh.ncols <= 0) continue;
    for (int r = 0; r < rt; ++r) {
      for (int c = 0; c < ct; ++c) {
        const int row0 = r * bm;
        int klo = 0, khi = sh.kdim;
        if (sh.tri == TRI_LOWER) khi = std::min(sh.kdim, row0 + bm);
        if (sh.tri == TRI_UPPER) klo = std::min(sh.kdim, row0);
        const int cols = std::min(cw, sh.ncols - c * cw);
        const int rows = std::min(bm, sh.m - row0);
        // SM clocks per k-block.  FP64: 2 DFMA/clk/SM; double-float: 13 FP32
        // instructions per multiply-add at 128 lanes/clk/SM.  A one-column
        // (GEMV) tile is bound by its tile load and barriers; a partial tile
        // of 2..48 columns runs the predicated path at about full-tile cost.
        const double per_col = (cost_model == COST_DF32) ? GEMM_BM * GEMM_BK * 13.0 / 128.0 : 0.5 * GEMM_BM * GEMM_BK;
        const double load = (cost_model == COST_DF32) ? 600.0 : 512.0;
        const int eff_cols = (cols == 1) ? 1 : (cols >= GEMM_BN - 15 ? cols : GEMM_BN);
        double cost = (cols == 1) ? per_col + 1500.0 : per_col * eff_cols + load;
        // tensor-core plan, per 16 k: 28 MMAs of 128 x 64 x 16 (~25 ns each on
        // one SM) against 42 KB of digit tiles; a GEMV k-block reads 16 KB
        if (tc) cost = (cols == 1) ? 300.0 : 1000.0;
        Tile t{o, row0, c * cw, klo / GEMM_BK, (khi + GEMM_BK - 1) / GEMM_BK, cost, cols == 1};
        tiles.push_back(t);
        flops += 2.0 * rows * cols * (double)(khi - klo);
        if (c == 0) {  // operator rows of this tile, once
          plan.alg_bytes += 8.0 * rows * (double)(khi - klo);
          plan.alg_op_bytes[o] += 8.0 * rows * (double)(khi - klo);
        }
      }
    }
  }
  for (int o = 0; o < plan.nops; ++o)  // X read once, C written once
    plan.alg_bytes += 8.0 * ((double)shapes[o].kdim + shapes[o].m) * std::max(0, shapes[o].ncols);
  plan.ntiles = (int)tiles.size();
  plan.total_out = outpos;
  plan.flops = flops;
  double W = 0;
  int64_t nkb = 0;
  for (auto& t : tiles) {
    W += t.cost_per_kb * (t.kb1 - t.kb0);
    nkb += t.kb1 - t.kb0;
  }
  const int C = (int)std::max<int64_t>(1, std::min<int64_t>(max_ctas, nkb));
  plan.nctas = C;
  std::vector<GemmSeg> segs;
  std::vector<int> seg_start(C + 1, 0);
  std::vector<std::vector<int>> tile_slots(tiles.size());
  // walk the linearised (tile, k-block) list; the CTA of an item is fixed by
  // the midpoint of its cost interval.  The tensor-core plan balances its
  // one-column (double-float GEMV) work and its tensor-core work as two
  // separate partitions and lists a CTA's GEMV segments first: its epilogue
  // warps run them while the copy and MMA warps stream the tensor-core tiles.
  std::vector<std::vector<GemmSeg>> per_cta(C);
  auto assign = [&](int pass) {
    double Wp = 0;
    for (auto& t : tiles)
      if (!tc || (pass == 0) == t.gemv) Wp += t.cost_per_kb * (t.kb1 - t.kb0);
    if (Wp <= 0) return;
    double cum = 0;
    int cur_cta = -1;
    // the tensor-core plan walks its GEMV tiles from the last op to the first:
    // the ops listed last (the R family) then share no CTA between their GEMV
    // rows and their digit tiles, both streamed from DRAM, while the first
    // ops' (B, Q: first-row and shared-tile reads from L2) land beside them
    const int nt = (int)tiles.size();
    for (int tj = 0; tj < nt; ++tj) {
      const int ti = (tc && pass == 0) ? nt - 1 - tj : tj;
      const Tile& t = tiles[ti];
      if (tc && (pass == 0) != t.gemv) continue;
      for (int kb = t.kb0; kb < t.kb1; ++kb) {
        const double mid = cum + 0.5 * t.cost_per_kb;
        cum += t.cost_per_kb;
        int cta = (int)std::floor(mid / Wp * C);
        cta = std::min(std::max(cta, 0), C - 1);
        auto& lst = per_cta[cta];
        const int k0 = kb * GEMM_BK;
        const int k1 = std::min(shapes[t.op].kdim, (kb + 1) * GEMM_BK);
        // tensor-core plan: exact segments of at most OZ_KMAX k; GEMV segments of
        // at most OZ_GEMV_K k (fine grains to interleave with the MMA segments)
        const int kcap = t.gemv ? OZ_GEMV_K : OZ_KMAX;
        if (!lst.empty() && lst.back().op == t.op && lst.back().row0 == t.row0 && lst.back().col0 == t.col0 &&
            lst.back().k1 == k0 && cur_cta == cta && (!tc || k1 - lst.back().k0 <= kcap)) {
          lst.back().k1 = k1;
        } else {
          lst.push_back(GemmSeg{t.op, t.row0, t.col0, k0, k1, ti /* tile id, slot assigned below */,
                                plan.col_width[t.op]});
        }
        cur_cta = cta;
      }
    }
  };
  // Tensor-core tiles in whole-tile chunks: a CTA whose k-range crossed a
  // tile boundary ran two accumulations in TMEM with a drain between them
  // (the MMAs wait for it) and a second drain at its end, and set the
  // launch's end.  Each tile t gets n_t chunks of near-equal k, with the
  // smallest longest chunk for which sum n_t <= C and every chunk fits one
  // exact segment; where no such split exists (more k per CTA than one
  // segment holds), the cost walk above cuts across tiles as before.
  auto assign_chunks = [&]() -> bool {
    std::vector<int> wide;
    int64_t longest = 0;
    for (int ti = 0; ti < (int)tiles.size(); ++ti)
      if (!tiles[ti].gemv) {
        wide.push_back(ti);
        longest = std::max<int64_t>(longest, tiles[ti].kb1 - tiles[ti].kb0);
      }
    if (wide.empty()) return true;
    const int64_t cap = OZ_KMAX / GEMM_BK;
    for (int64_t L = 1; L <= std::min(longest, cap); ++L) {
      int64_t used = 0;
      for (int ti : wide) used += (tiles[ti].kb1 - tiles[ti].kb0 + L - 1) / L;
      if (used > C) continue;
      int cta = 0;
      for (int ti : wide) {
        const Tile& t = tiles[ti];
        const int64_t len = t.kb1 - t.kb0, n = (len + L - 1) / L;
        for (int64_t q = 0; q < n; ++q, ++cta) {
          const int64_t b0 = t.kb0 + len * q / n, b1 = t.kb0 + len * (q + 1) / n;
          if (b1 <= b0) continue;
          per_cta[cta].push_back(GemmSeg{t.op, t.row0, t.col0, (int)b0 * GEMM_BK,
                                         std::min(shapes[t.op].kdim, (int)b1 * GEMM_BK), ti, plan.col_width[t.op]});
        }
      }
      return true;
    }
    return false;
  };
  assign(0);
  if (tc) {
    if (!assign_chunks()) assign(1);
    // order of a CTA's list: g_0, T_0, g_1, T_1, ..., g_{n-1}, T_{n-1}, with the
    // GEMV segments g_i sized like the tensor-core segment T_i.  The epilogue
    // warps run g_i while the MMAs of T_i proceed, then drain T_i just before
    // T_{i+1} needs the accumulators.
    for (auto& lst : per_cta) {
      std::vector<GemmSeg> G, T;
      for (auto& sg : lst) (tiles[sg.slot].gemv ? G : T).push_back(sg);
      if (T.empty() || G.empty()) continue;
      double tkb = 0;
      for (auto& sg : T) tkb += sg.k1 - sg.k0;
      double gk = 0;
      for (auto& sg : G) gk += sg.k1 - sg.k0;
      std::vector<GemmSeg> out;
      size_t gi = 0;
      double done_t = 0, done_g = 0;
      for (auto& sg : T) {
        done_t += sg.k1 - sg.k0;
        const double target = gk * done_t / tkb;  // GEMV k to have been issued by the end of this gap
        while (gi < G.size() && done_g + 0.5 * (G[gi].k1 - G[gi].k0) <= target) {
          done_g += G[gi].k1 - G[gi].k0;
          out.push_back(G[gi++]);
        }
        out.push_back(sg);
      }
      while (gi < G.size()) out.push_back(G[gi++]);
      lst.swap(out);
    }
  }
  (void)W;
  int slot = 0;
  for (int c = 0; c < C; ++c) {
    seg_start[c] = (int)segs.size();
    for (auto sg : per_cta[c]) {
      const int ti = sg.slot;
      sg.slot = slot++;
      tile_slots[ti].push_back(sg.slot);
      segs.push_back(sg);
    }
  }
  seg_start[C] = (int)segs.size();
  plan.nslots = slot;
  if (tc) {
    double bytes = 0, mma = 0, dbytes = 0;
    for (int o = 0; o < plan.nops; ++o)  // X digits (once per op; the row tiles re-read them from L2)
      dbytes += 2.0 * (double)oz_x_elems(shapes[o].kdim, shapes[o].ncols);
    for (const GemmSeg& sg : segs) {
      const OpShape& sh = shapes[sg.op];
      const int cols = std::min(sg.colw, sh.ncols - sg.col0);
      const int rows = std::min(bm, sh.m - sg.row0);
      WC4D_CHECK(sg.k1 - sg.k0 <= (cols >= 2 ? OZ_KMAX : OZ_GEMV_K), WC4D_ERR_ARG,
                 "internal: tensor-core plan segment longer than its exact / GEMV limit");
      const int kbs = (sg.k1 + OZ_BK - 1) / OZ_BK - sg.k0 / OZ_BK;
      if (cols >= 2) {
        dbytes += (double)kbs * 2.0 * OZ_DIGITS * OZ_A_TILE;
        plan.tc_digit_op_bytes[sg.op] += (double)kbs * 2.0 * OZ_DIGITS * OZ_A_TILE;
        bytes += 8.0 * rows * cols;
        mma += (double)kbs * (OZ_DIGITS * (OZ_DIGITS + 1) / 2) * 2.0 * OZ_BM * OZ_BN * OZ_BK;
      } else {
        bytes += 8.0 * rows * (double)(sg.k1 - sg.k0) + 8.0 * (sg.k1 - sg.k0) + 8.0 * rows;
        plan.tc_gemv_op_bytes[sg.op] += 8.0 * rows * (double)(sg.k1 - sg.k0);
      }
    }
    plan.tc_bytes = bytes + dbytes;
    plan.tc_digit_bytes = dbytes;
    plan.tc_mma_flops = mma;
  }
  // slots of a tile in k order (segments were appended in k order per CTA and
  // CTAs in increasing order, which is also increasing k within a tile)
  std::vector<int> tstart(tiles.size() + 1, 0), tslots;
  for (size_t i = 0; i < tiles.size(); ++i) {
    tstart[i] = (int)tslots.size();
    for (int sl : tile_slots[i]) tslots.push_back(sl);
  }
  tstart[tiles.size()] = (int)tslots.size();
  if (tslots.empty()) tslots.push_back(0);
  if (segs.empty()) segs.push_back(GemmSeg{0, 0, 0, 0, 0, 0, 1});
  auto arrays = std::make_shared<PlanArrays>();
  plan.owner = arrays;
  WC4D_CUDA(cudaMalloc(&arrays->p[0], sizeof(int) * seg_start.size()));
  WC4D_CUDA(cudaMalloc(&arrays->p[1], sizeof(GemmSeg) * segs.size()));
  WC4D_CUDA(cudaMalloc(&arrays->p[2], sizeof(int) * tstart.size()));
  WC4D_CUDA(cudaMalloc(&arrays->p[3], sizeof(int) * tslots.size()));
  plan.d_seg_start = (int*)arrays->p[0];
  plan.d_segs = (GemmSeg*)arrays->p[1];
  plan.d_tile_start = (int*)arrays->p[2];
  plan.d_tile_slots = (int*)arrays->p[3];
  WC4D_CUDA(cudaMemcpy(plan.d_seg_start, seg_start.data(), sizeof(int) * seg_start.size(), cudaMemcpyHostToDevice));
  WC4D_CUDA(cudaMemcpy(plan.d_segs, segs.data(), sizeof(GemmSeg) * segs.size(), cudaMemcpyHostToDevice));
  WC4D_CUDA(cudaMemcpy(plan.d_tile_start, tstart.data(), sizeof(int) * tstart.size(), cudaMemcpyHostToDevice));
  WC4D_CUDA(cudaMemcpy(plan.d_tile_slots, tslots.data(), sizeof(int) * tslots.size(), cudaMemcpyHostToDevice));
  std::lock_guard<std::mutex> lk(g_plan_mu);
  if (plan_cache().size() >= PLAN_CACHE_MAX) plan_cache().clear();  // live problems keep their plans
  plan_cache().emplace(key, plan);
}

// ---------------------------------------------------------------- kernels
// 256 threads; thread (tx, ty) owns rows row0 + tx + 16 i and columns
// col0 + ty + 16 j (i, j < 4): conflict-free shared reads and coalesced
// column-major partial stores.  The next k-block is prefetched into registers
// while the current one is multiplied.  A one-column tile (a single time level,
// e.g. B v1_0) switches to a GEMV mapping: every thread takes one row and a
// quarter of the k-block, so all four SM sub-partitions share the work.
template <typename T>
__global__ void __launch_bounds__(256) gemm_streamk_kernel(GemmOpsT<T> ops, const GemmSeg* __restrict__ segs,
                                                           const int* __restrict__ seg_start, T* __restrict__ partial,
                                                           const int* __restrict__ done, int* ran) {
  if (done != nullptr && *(volatile const int*)done) return;
  if (ran != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *ran = 1;
  __shared__ T As[GEMM_BK][GEMM_BM + 1];
  __shared__ T Xs[GEMM_BK][GEMM_BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  constexpr int LA = (GEMM_BM * GEMM_BK) / 256;
  constexpr int LX = (GEMM_BN * GEMM_BK) / 256;
  const int sbeg = seg_start[blockIdx.x], send = seg_start[blockIdx.x + 1];
  for (int si = sbeg; si < send; ++si) {
    const GemmSeg sg = segs[si];
    const GemmOpT<T> op = ops.op[sg.op];
    const int ncv = min(sg.colw, op.ncols - sg.col0);  // columns present in this tile
    T ra[LA], rx[LX];
    auto fetch = [&](int k) {
#pragma unroll
      for (int q = 0; q < LA; ++q) {
        const int e = tid + 256 * q;
        const int kk = e % GEMM_BK, ii = e / GEMM_BK;
        const int gi = sg.row0 + ii, gk = k + kk;
        ra[q] = (gi < op.m && gk < sg.k1) ? op.At[gk + (int64_t)gi * op.lda] : T(0);
      }
#pragma unroll
      for (int q = 0; q < LX; ++q) {
        const int e = tid + 256 * q;
        const int kk = e % GEMM_BK, cc = e / GEMM_BK;
        const int gk = k + kk;
        rx[q] = (cc < ncv && gk < sg.k1) ? op.X[gk + (int64_t)(sg.col0 + cc) * op.ldx] : T(0);
      }
    };
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    fetch(sg.k0);
    for (int k = sg.k0; k < sg.k1; k += GEMM_BK) {
#pragma unroll
      for (int q = 0; q < LA; ++q) {
        const int e = tid + 256 * q;
        As[e % GEMM_BK][e / GEMM_BK] = ra[q];
      }
#pragma unroll
      for (int q = 0; q < LX; ++q) {
        const int e = tid + 256 * q;
        Xs[e % GEMM_BK][e / GEMM_BK] = rx[q];
      }
      __syncthreads();
      if (k + GEMM_BK < sg.k1) fetch(k + GEMM_BK);
      if (ncv == 1) {
        // GEMV mapping: row tid % 64, k-slice tid / 64
        const int r = tid & 63, q0 = tid >> 6;
#pragma unroll
        for (int kk = q0; kk < GEMM_BK; kk += 4) acc[0][0] = fma(As[kk][r], Xs[kk][0], acc[0][0]);
      } else if (ncv >= GEMM_BN - 15) {
#pragma unroll
        for (int kk = 0; kk < GEMM_BK; ++kk) {
          T a[4], x[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
          for (int j = 0; j < 4; ++j) x[j] = Xs[kk][ty + 16 * j];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], x[j], acc[i][j]);
        }
      } else if (ty < ncv) {
#pragma unroll
        for (int kk = 0; kk < GEMM_BK; ++kk) {
          T a[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (ty + 16 * j < ncv) {
              const T x = Xs[kk][ty + 16 * j];
#pragma unroll
              for (int i = 0; i < 4; ++i) acc[i][j] = fma(a[i], x, acc[i][j]);
            }
          }
        }
      }
      __syncthreads();
    }
    T* dst = partial + (int64_t)sg.slot * (GEMM_BM * GEMM_BN);
    if (ncv == 1) {
      // combine the four k-slices of each row (reuses As as scratch)
      T* red = &As[0][0];
      red[tid] = acc[0][0];
      __syncthreads();
      if (tid < GEMM_BM) dst[tid] = (red[tid] + red[tid + 64]) + (red[tid + 128] + red[tid + 192]);
      __syncthreads();
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) dst[(ty + 16 * j) * GEMM_BM + tx + 16 * i] = acc[i][j];
    }
  }
}

// ------------------------------------------------- double-float products
// df_mac / df_mac2 (common.cuh): FP64-class multiply-add on the FP32 pipe.

__global__ void __launch_bounds__(256) gemm_streamk_df32_kernel(GemmOpsT<double> ops,
                                                                const GemmSeg* __restrict__ segs,
                                                                const int* __restrict__ seg_start,
                                                                double* __restrict__ partial,
                                                                const int* __restrict__ done, int* ran) {
  if (done != nullptr && *(volatile const int*)done) return;
  if (ran != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *ran = 1;
  __shared__ float Ah[GEMM_BK][GEMM_BM + 1];
  __shared__ float Al[GEMM_BK][GEMM_BM + 1];
  __shared__ float Xh[GEMM_BK][GEMM_BN + 1];
  __shared__ float Xl[GEMM_BK][GEMM_BN + 1];
  __shared__ double red[256];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  constexpr int LA = (GEMM_BM * GEMM_BK) / 256;
  constexpr int LX = (GEMM_BN * GEMM_BK) / 256;
  const int sbeg = seg_start[blockIdx.x], send = seg_start[blockIdx.x + 1];
  for (int si = sbeg; si < send; ++si) {
    const GemmSeg sg = segs[si];
    const GemmOpT<double> op = ops.op[sg.op];
    const int ncv = min(sg.colw, op.ncols - sg.col0);
    float rah[LA], ral[LA], rxh[LX], rxl[LX];
    auto fetch = [&](int k) {
#pragma unroll
      for (int q = 0; q < LA; ++q) {
        const int e = tid + 256 * q;
        const int kk = e % GEMM_BK, ii = e / GEMM_BK;
        const int gi = sg.row0 + ii, gk = k + kk;
        const bool in = (gi < op.m && gk < sg.k1);
        const int64_t idx = gk + (int64_t)gi * op.lda;
        rah[q] = in ? op.Ah[idx] : 0.f;
        ral[q] = in ? op.Al[idx] : 0.f;
      }
#pragma unroll
      for (int q = 0; q < LX; ++q) {
        const int e = tid + 256 * q;
        const int kk = e % GEMM_BK, cc = e / GEMM_BK;
        const int gk = k + kk;
        const bool in = (cc < ncv && gk < sg.k1);
        const int64_t idx = gk + (int64_t)(sg.col0 + cc) * op.m;  // split X is dense, ld = m
        rxh[q] = in ? op.Xh[idx] : 0.f;
        rxl[q] = in ? op.Xl[idx] : 0.f;
      }
    };
    float s[4][4], c[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) s[i][j] = c[i][j] = 0.f;
    fetch(sg.k0);
    for (int k = sg.k0; k < sg.k1; k += GEMM_BK) {
#pragma unroll
      for (int q = 0; q < LA; ++q) {
        const int e = tid + 256 * q;
        Ah[e % GEMM_BK][e / GEMM_BK] = rah[q];
        Al[e % GEMM_BK][e / GEMM_BK] = ral[q];
      }
#pragma unroll
      for (int q = 0; q < LX; ++q) {
        const int e = tid + 256 * q;
        Xh[e % GEMM_BK][e / GEMM_BK] = rxh[q];
        Xl[e % GEMM_BK][e / GEMM_BK] = rxl[q];
      }
      __syncthreads();
      if (k + GEMM_BK < sg.k1) fetch(k + GEMM_BK);
      if (ncv == 1) {
        const int r = tid & 63, q0 = tid >> 6;
#pragma unroll
        for (int kk = q0; kk < GEMM_BK; kk += 4) df_mac(s[0][0], c[0][0], Ah[kk][r], Al[kk][r], Xh[kk][0], Xl[kk][0]);
      } else if (ncv >= GEMM_BN - 15) {
        // output pairs (j, j+1) share one paired instruction stream
        float2 s2[4][2], c2[4][2];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            s2[i][q] = make_float2(s[i][2 * q], s[i][2 * q + 1]);
            c2[i][q] = make_float2(c[i][2 * q], c[i][2 * q + 1]);
          }
#pragma unroll 4
        for (int kk = 0; kk < GEMM_BK; ++kk) {
          float ah[4], al[4];
          float2 xh[2], xl[2];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            ah[i] = Ah[kk][tx + 16 * i];
            al[i] = Al[kk][tx + 16 * i];
          }
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            xh[q] = make_float2(Xh[kk][ty + 32 * q], Xh[kk][ty + 32 * q + 16]);
            xl[q] = make_float2(Xl[kk][ty + 32 * q], Xl[kk][ty + 32 * q + 16]);
          }
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int q = 0; q < 2; ++q)
              df_mac2(s2[i][q], c2[i][q], make_float2(ah[i], ah[i]), make_float2(al[i], al[i]), xh[q], xl[q]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            s[i][2 * q] = s2[i][q].x;
            s[i][2 * q + 1] = s2[i][q].y;
            c[i][2 * q] = c2[i][q].x;
            c[i][2 * q + 1] = c2[i][q].y;
          }
      } else if (ty < ncv) {
        for (int kk = 0; kk < GEMM_BK; ++kk) {
          float ah[4], al[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            ah[i] = Ah[kk][tx + 16 * i];
            al[i] = Al[kk][tx + 16 * i];
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (ty + 16 * j < ncv) {
              const float xh = Xh[kk][ty + 16 * j], xl = Xl[kk][ty + 16 * j];
#pragma unroll
              for (int i = 0; i < 4; ++i) df_mac(s[i][j], c[i][j], ah[i], al[i], xh, xl);
            }
          }
        }
      }
      __syncthreads();
    }
    // partial tiles stay double-float pairs (s, c): the FP64 conversion is done
    // once per output by the reduce kernel, off GB300's 1/64-rate FP64 pipe here
    float2* dst = reinterpret_cast<float2*>(partial) + (int64_t)sg.slot * (GEMM_BM * GEMM_BN);
    if (ncv == 1) {
      float2* red2 = reinterpret_cast<float2*>(red);
      float h, l;
      two_sum(s[0][0], c[0][0], h, l);
      red2[tid] = make_float2(h, l);
      __syncthreads();
      if (tid < GEMM_BM)
        dst[tid] = df_add(df_add(red2[tid], red2[tid + 64]), df_add(red2[tid + 128], red2[tid + 192]));
      __syncthreads();
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) dst[(ty + 16 * j) * GEMM_BM + tx + 16 * i] = make_float2(s[i][j], c[i][j]);
    }
  }
}

struct ReduceMeta {
  int nops;
  int tile_base[GEMM_MAX_OPS];
  int col_tiles[GEMM_MAX_OPS];
  int col_width[GEMM_MAX_OPS];
  int m[GEMM_MAX_OPS];
  int ncols[GEMM_MAX_OPS];
  int64_t out_base[GEMM_MAX_OPS];
  int64_t total;
  int pairs;  // partials are double-float pairs (s, c) written by the DF32 kernel
  int bm;     // rows per tile / partial slot
};

template <typename T>
__global__ void __launch_bounds__(256, 6) gemm_reduce_kernel(ReduceMeta meta, EpisT<T> epis, const T* __restrict__ partial,
                                                          const int* __restrict__ tile_start,
                                                          const int* __restrict__ tile_slots, ModelDev md,
                                                          const int* __restrict__ obs, const int* __restrict__ done) {
  pdl_wait();
  pdl_trigger();
  if (done != nullptr && *(volatile const int*)done) return;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < meta.total;
       g += (int64_t)gridDim.x * blockDim.x) {
    int o = 0;
    while (o + 1 < meta.nops && g >= meta.out_base[o + 1]) ++o;
    // 32-bit index arithmetic: one op's outputs m * ncols < 2^31 (checked by the
    // plan); 64-bit division per element is a long emulated sequence
    const int e = (int)(g - meta.out_base[o]);
    const int m = meta.m[o];
    const int r = e % m, c = e / m;
    const int cw = meta.col_width[o];
    const int bm = meta.bm;
    const int tile = meta.tile_base[o] + (r / bm) * meta.col_tiles[o] + c / cw;
    const int off = (c % cw) * bm + (r % bm);
    const int64_t slot_elems = (int64_t)bm * GEMM_BN;
    T acc = T(0);
    // the epilogue operands do not depend on the partials: load them first so
    // their latency overlaps the slot-index / partial chain below
    const EpiT<T>& ep = epis.e[o];
    T pre = T(0);
    switch (ep.mode) {
      case EPI_SADDLE_C1: {
        const int t = c + ep.t0;
        const int s = md.s;
        pre = ep.v3[(int64_t)t * s + r];
        if (t >= 1) pre -= model_apply<T>(md, t, ep.v3 + (int64_t)(t - 1) * s, r);
        break;
      }
      case EPI_SADDLE_C2:
        pre = ep.v3[(int64_t)(c + ep.t0) * md.s + obs[r]];
        break;
      case EPI_SUB_FROM:
        pre = ep.Y[r + (int64_t)c * ep.ldc];
        break;
      default:
        break;
    }
    // slots in batches of 8: the slot indices, then the partials, are loaded
    // together (independent loads in flight) and summed in slot order
    constexpr int RB = 8;
    const int q0 = tile_start[tile], q1 = tile_start[tile + 1];
    if (sizeof(T) == 8 && meta.pairs) {
      const float2* pp = reinterpret_cast<const float2*>(partial);
      float2 a2 = make_float2(0.f, 0.f);
      for (int qb = q0; qb < q1; qb += RB) {
        int sl[RB];
        float2 v[RB];
#pragma unroll
        for (int u = 0; u < RB; ++u) sl[u] = (qb + u < q1) ? tile_slots[qb + u] : -1;
#pragma unroll
        for (int u = 0; u < RB; ++u) v[u] = sl[u] >= 0 ? pp[(int64_t)sl[u] * slot_elems + off] : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < RB; ++u) {
          if (sl[u] < 0) break;
          float h, l;
          two_sum(v[u].x, v[u].y, h, l);
          a2 = df_add(a2, make_float2(h, l));
        }
      }
      acc = T((double)a2.x + (double)a2.y);
    } else {
      for (int qb = q0; qb < q1; qb += RB) {
        int sl[RB];
        T v[RB];
#pragma unroll
        for (int u = 0; u < RB; ++u) sl[u] = (qb + u < q1) ? tile_slots[qb + u] : -1;
#pragma unroll
        for (int u = 0; u < RB; ++u) v[u] = sl[u] >= 0 ? partial[(int64_t)sl[u] * slot_elems + off] : T(0);
#pragma unroll
        for (int u = 0; u < RB; ++u) {
          if (sl[u] < 0) break;
          acc += v[u];
        }
      }
    }
    T val;
    switch (ep.mode) {
      case EPI_SADDLE_C1:
      case EPI_SADDLE_C2:
        val = acc + pre;
        break;
      case EPI_SUB_FROM:
        val = pre - acc;
        break;
      case EPI_NEG_STORE:
        val = -acc;
        break;
      default:
        val = acc;
    }
    ep.C[r + (int64_t)c * ep.ldc] = val;
    if (sizeof(T) == 8 && ep.Ch != nullptr) {
      const float h = (float)val;
      ep.Ch[r + (int64_t)c * ep.ldc] = h;
      ep.Cl[r + (int64_t)c * ep.ldc] = (float)((double)val - (double)h);
    }
  }
}

template <typename T>
static void launch_products(const GemmPlan& plan, const GemmOpsT<T>& ops, T* partial, const int* done,
                            cudaStream_t st) {
  int* ran = prof_begin(sizeof(T) == 8 ? PROF_GEMM : PROF_GEMM32, plan.flops, st);
  gemm_streamk_kernel<T><<<plan.nctas, 256, 0, st>>>(ops, plan.d_segs, plan.d_seg_start, partial, done, ran);
  WC4D_LAUNCH_CHECK();
  if (ran) prof_end(st);
}
template <>
void launch_products<double>(const GemmPlan& plan, const GemmOpsT<double>& ops, double* partial, const int* done,
                             cudaStream_t st) {
  if (ops.tc) {
    // with nd of the 7 digits: the digit tiles' bytes and the digit products shrink
    const int nd = ops.ndig;
    double bytes = plan.tc_bytes - plan.tc_digit_bytes * (1.0 - nd / (double)OZ_DIGITS);
    const double mma = plan.tc_mma_flops * (nd * (nd + 1) / 2) / (double)(OZ_DIGITS * (OZ_DIGITS + 1) / 2);
    double alg = plan.alg_bytes;
    for (int o = 0; o < plan.nops; ++o) {
      const GemmOpT<double>& op = ops.op[o];
      const OpShape& sh = plan.shape[o];
      const bool wide = oz_wide_tiles(sh.ncols) > 0, gemv = oz_gemv_col(sh.ncols) >= 0;
      // a Toeplitz operator's GEMV rows come from its first row: 8 B per k
      // instead of 8 B per entry
      const double row = 8.0 * sh.kdim;
      if (op.Th) bytes += row - plan.tc_gemv_op_bytes[o];
      // its shared digit tiles: each distinct tile once, the rest L2 re-reads
      if (op.toep_tiles) {
        const int64_t nkb = (sh.kdim + OZ_BK - 1) / OZ_BK, rt = (sh.m + OZ_BM - 1) / OZ_BM;
        const double distinct = (double)std::min<int64_t>(rt * nkb, nkb + (OZ_BM / OZ_BK) * (rt - 1));
        bytes -= (plan.tc_digit_op_bytes[o] - distinct * 2.0 * OZ_DIGITS * OZ_A_TILE) * (nd / (double)OZ_DIGITS);
      }
      // with every tile of the op served from the first row or the shared
      // tiles, the row is the op's floor too
      if ((op.Th || !gemv) && (op.toep_tiles || !wide) && (op.Th || op.toep_tiles))
        alg += row - plan.alg_op_bytes[o];
    }
    int* ran = prof_begin(PROF_GEMMTC, plan.flops, st, bytes, mma, alg);
    launch_gemm_tc(ops, plan.d_segs, plan.d_seg_start, plan.nctas, partial, done, ran, ops.err, st);
    if (ran) prof_end(st);
    return;
  }
  const bool df = ops.df32 != 0;
  int* ran = prof_begin(df ? PROF_GEMMDF : PROF_GEMM, plan.flops, st);
  if (df)
    gemm_streamk_df32_kernel<<<plan.nctas, 256, 0, st>>>(ops, plan.d_segs, plan.d_seg_start, partial, done, ran);
  else
    gemm_streamk_kernel<double><<<plan.nctas, 256, 0, st>>>(ops, plan.d_segs, plan.d_seg_start, partial, done, ran);
  WC4D_LAUNCH_CHECK();
  if (ran) prof_end(st);
}

// resident CTAs of the reduction kernel (all SMs)
template <typename T>
static int reduce_resident_ctas() {
  static std::atomic<int> cached{0};  // one per instance; host threads may race to fill it, all with the same value
  if (const int c = cached.load(std::memory_order_relaxed)) return c;
  int dev = 0, sms = 0, per = 0;
  WC4D_CUDA(cudaGetDevice(&dev));
  WC4D_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  WC4D_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, gemm_reduce_kernel<T>, 256, 0));
  const int c = std::max(1, sms * std::max(1, per));
  cached.store(c, std::memory_order_relaxed);
  return c;
}

template <typename T>
void gemm_run(const GemmPlan& plan, const GemmOpsT<T>& ops, const EpisT<T>& epis, T* partial, const ModelDev& model,
              const int* obs, const int* done, cudaStream_t st) {
  if (plan.total_out == 0) return;
  if (plan.nslots > 0) launch_products<T>(plan, ops, partial, done, st);
  ReduceMeta meta;
  meta.nops = plan.nops;
  for (int o = 0; o < GEMM_MAX_OPS; ++o) {
    meta.tile_base[o] = o < plan.nops ? plan.tile_base[o] : 0;
    meta.col_tiles[o] = o < plan.nops ? plan.col_tiles[o] : 1;
    meta.col_width[o] = o < plan.nops ? std::max(1, plan.col_width[o]) : 1;
    meta.m[o] = o < plan.nops ? std::max(1, plan.shape[o].m) : 1;
    meta.ncols[o] = o < plan.nops ? plan.shape[o].ncols : 0;
    meta.out_base[o] = o < plan.nops ? plan.out_base[o] : plan.total_out;
  }
  meta.total = plan.total_out;
  meta.pairs = (sizeof(T) == 8 && (ops.df32 != 0 || ops.tc != 0)) ? 1 : 0;
  meta.bm = plan.bm;
  WC4D_CHECK(plan.bm == GEMM_BM || (sizeof(T) == 8 && ops.tc), WC4D_ERR_ARG,
             "internal: tensor-core plan run without the tensor-core operands");
  // at most one resident wave (six 256-thread CTAs per SM): a few CTAs past it
  // would run as a second wave of their own and nearly double the launch
  const int64_t nb = std::min<int64_t>((plan.total_out + 255) / 256, reduce_resident_ctas<T>());
  WC4D_CUDA(launch_pdl(gemm_reduce_kernel<T>, dim3((unsigned)nb), dim3(256), 0, st, meta, epis, (const T*)partial,
                       (const int*)plan.d_tile_start, (const int*)plan.d_tile_slots, model, obs, done));
  WC4D_LAUNCH_CHECK();
}

int gemm_resident_ctas(bool df32) {
  // set by whichever host thread (a batched solve's workers) asks first; all compute the same value
  static std::atomic<int> cached[2]{};
  if (const int c = cached[df32].load(std::memory_order_relaxed)) return c;
  int dev = 0, sms = 0, per = 0, per32 = 0;
  WC4D_CUDA(cudaGetDevice(&dev));
  WC4D_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (df32)
    WC4D_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, gemm_streamk_df32_kernel, 256, 0));
  else
    WC4D_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, gemm_streamk_kernel<double>, 256, 0));
  // the FP32 instance shares the schedule; use the smaller residency of the two
  WC4D_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per32, gemm_streamk_kernel<float>, 256, 0));
  const int c = std::max(1, sms * std::max(1, std::min(per, per32)));
  cached[df32].store(c, std::memory_order_relaxed);
  return c;
}

template void gemm_run<double>(const GemmPlan&, const GemmOpsT<double>&, const EpisT<double>&, double*,
                               const ModelDev&, const int*, const int*, cudaStream_t);
template void gemm_run<float>(const GemmPlan&, const GemmOpsT<float>&, const EpisT<float>&, float*, const ModelDev&,
                              const int*, const int*, cudaStream_t);

}  // namespace wc4d
