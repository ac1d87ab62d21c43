// Kernel-level timing and launch counting (measurement support).
#include <atomic>

#include "runtime.h"

namespace compar {

static std::atomic<int64_t> g_launches{0};

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

cudaEvent_t KernelProfiler::begin(cudaStream_t s) {
  if (!on) return nullptr;
  cudaEvent_t e = nullptr;
  if (!pool.empty()) {
    e = pool.back();
    pool.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    return nullptr;
  }
  cudaEventRecord(e, s);
  return e;
}

void KernelProfiler::end(cudaEvent_t a, cudaStream_t s, int v) {
  if (!a) return;
  cudaEvent_t b = nullptr;
  if (!pool.empty()) {
    b = pool.back();
    pool.pop_back();
  } else if (cudaEventCreate(&b) != cudaSuccess) {
    pool.push_back(a);
    return;
  }
  cudaEventRecord(b, s);
  pend.push_back(Pend{a, b, v});
  if (pend.size() >= 8192) resolve();
}

void KernelProfiler::resolve() {
  for (auto& p : pend) {
    float ms = 0;
    if (cudaEventSynchronize(p.b) == cudaSuccess &&
        cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess && p.v >= 0 && p.v < kSlots) {
      total_ms[p.v] += ms;
      launches[p.v] += 1;
    }
    pool.push_back(p.a);
    pool.push_back(p.b);
  }
  pend.clear();
}

void KernelProfiler::reset() {
  resolve();
  for (int i = 0; i < kSlots; ++i) {
    total_ms[i] = 0;
    launches[i] = 0;
  }
}

void KernelProfiler::release() {
  resolve();
  for (auto e : pool) cudaEventDestroy(e);
  pool.clear();
}

}  // namespace compar

using namespace compar;

extern "C" {

int compar_profile_enable(compar_ctx_t ctx, int on) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  if (!ctx) return COMPAR_ERR_INVALID;
  ctx->prof.on = on != 0;
  if (!on) ctx->prof.resolve();
  return COMPAR_OK;
}

int compar_profile_read(compar_ctx_t ctx, int variant, double* kernel_ms, int64_t* launches) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  if (!ctx || variant < 0 || variant >= KernelProfiler::kSlots || !kernel_ms || !launches)
    return COMPAR_ERR_INVALID;
  ctx->prof.resolve();
  *kernel_ms = ctx->prof.total_ms[variant];
  *launches = ctx->prof.launches[variant];
  return COMPAR_OK;
}

int compar_profile_reset(compar_ctx_t ctx) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  if (!ctx) return COMPAR_ERR_INVALID;
  ctx->prof.reset();
  return COMPAR_OK;
}

int64_t compar_launch_count(void) { return launch_count(); }

}  // extern "C"
