// Launch counting and the opt-in kernel profile behind wc4d_get_stats.
#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace wc4d {

static std::atomic<int64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {
struct Rec {
  cudaEvent_t e0, e1;
  int cls;
  double work;
  int flag;
  double work2, work3, work4;
};
struct Profile {
  std::mutex mu;
  bool on = false;
  int* d_flags = nullptr;
  int cap = 0;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  Rec* open = nullptr;
};
Profile& prof() {
  static Profile p;
  return p;
}
cudaEvent_t get_event(Profile& p) {
  if (!p.pool.empty()) {
    cudaEvent_t e = p.pool.back();
    p.pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  WC4D_CUDA(cudaEventCreate(&e));
  return e;
}
}  // namespace

bool prof_enabled() { return prof().on; }

int* prof_begin(int cls, double work, cudaStream_t st, double work2, double work3, double work4) {
  Profile& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  if (!p.on || (int)p.recs.size() >= p.cap) return nullptr;
  // the flag slot is zero: slots are cleared when allocated and on every reset
  Rec r{get_event(p), get_event(p), cls, work, (int)p.recs.size(), work2, work3, work4};
  WC4D_CUDA(cudaEventRecord(r.e0, st));
  p.recs.push_back(r);
  return p.d_flags + r.flag;
}

void prof_end(cudaStream_t st) {
  Profile& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  if (!p.on || p.recs.empty()) return;
  WC4D_CUDA(cudaEventRecord(p.recs.back().e1, st));
}

}  // namespace wc4d

extern "C" {

void wc4d_set_profiling(int32_t enable) {
  using namespace wc4d;
  Profile& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  if (enable && !p.d_flags) {
    p.cap = 1 << 20;
    if (cudaMalloc(&p.d_flags, sizeof(int) * p.cap) != cudaSuccess ||
        cudaMemset(p.d_flags, 0, sizeof(int) * p.cap) != cudaSuccess) {
      cudaFree(p.d_flags);
      p.d_flags = nullptr;
      p.cap = 0;
      return;
    }
  }
  p.on = enable != 0 && p.d_flags != nullptr;
}

void wc4d_reset_stats(void) {
  using namespace wc4d;
  Profile& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  cudaDeviceSynchronize();
  if (p.d_flags && !p.recs.empty()) cudaMemset(p.d_flags, 0, sizeof(int) * p.recs.size());
  for (auto& r : p.recs) {
    p.pool.push_back(r.e0);
    p.pool.push_back(r.e1);
  }
  p.recs.clear();
  g_launches.store(0);
}

int wc4d_get_stats(wc4d_stats* out) {
  using namespace wc4d;
  if (!out) return WC4D_ERR_ARG;
  Profile& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  *out = wc4d_stats{};
  out->launches = g_launches.load();
  if (p.recs.empty()) return WC4D_OK;
  if (cudaDeviceSynchronize() != cudaSuccess) return WC4D_ERR_CUDA;
  std::vector<int> flags(p.recs.size());
  if (cudaMemcpy(flags.data(), p.d_flags, sizeof(int) * flags.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
    return WC4D_ERR_CUDA;
  for (size_t i = 0; i < p.recs.size(); ++i) {
    if (!flags[i]) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.recs[i].e0, p.recs[i].e1) != cudaSuccess) continue;
    if (p.recs[i].cls == PROF_GEMM) {
      out->gemm_ms += ms;
      out->gemm_flops += p.recs[i].work;
      out->gemm_launches += 1;
    } else if (p.recs[i].cls == PROF_GEMMDF) {
      out->gemmdf_ms += ms;
      out->gemmdf_flops += p.recs[i].work;
      out->gemmdf_launches += 1;
    } else if (p.recs[i].cls == PROF_GEMMTC) {
      out->gemmtc_ms += ms;
      out->gemmtc_flops += p.recs[i].work;
      out->gemmtc_bytes += p.recs[i].work2;
      out->gemmtc_mma_flops += p.recs[i].work3;
      out->gemmtc_alg_bytes += p.recs[i].work4;
      out->gemmtc_launches += 1;
    } else if (p.recs[i].cls == PROF_CIRC) {
      out->circ_ms += ms;
      out->circ_flops += p.recs[i].work;
      out->circ_bytes += p.recs[i].work2;
      out->circ_launches += 1;
    } else if (p.recs[i].cls == PROF_PERTIME) {
      out->pt_ms += ms;
      out->pt_bytes += p.recs[i].work;
      out->pt_launches += 1;
    } else if (p.recs[i].cls == PROF_GEMM32) {
      out->gemm32_ms += ms;
      out->gemm32_flops += p.recs[i].work;
      out->gemm32_launches += 1;
    } else {
      out->orth_ms += ms;
      out->orth_bytes += p.recs[i].work;
      out->orth_moved_bytes += p.recs[i].work2 > 0.0 ? p.recs[i].work2 : p.recs[i].work;
      out->orth_launches += 1;
    }
  }
  return WC4D_OK;
}

}  // extern "C"
