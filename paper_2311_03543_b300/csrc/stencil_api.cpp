// C ABI of the thermal-stencil component and its variant selection: the
// same runtime roles as for GEMM (registry with support rules, forced
// variant, decision cache, history table fed by measurements, roofline
// prior), on a second interface.  Every stencil variant computes the same
// rounded operations, so the error model has nothing to decide here: the
// selection is by time alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "runtime.h"

namespace compar {
namespace {

const char* kStencilNames[] = {"stencil-naive", "stencil-tiled", "stencil-tma"};
static_assert(sizeof(kStencilNames) / sizeof(kStencilNames[0]) == COMPAR_S_COUNT,
              "one name per stencil variant");

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

bool params_ok(const compar_stencil_params_t* p) {
  return p && std::isfinite(p->c) && std::isfinite(p->gx) && std::isfinite(p->gy) &&
         std::isfinite(p->gz) && std::isfinite(p->amb);
}

bool overlaps(const void* a, const void* b, size_t bytes) {
  const auto x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + bytes && y < x + bytes;
}

// Roofline prior (ms).  NAIVE: per step, read T and P and write T (12 bytes
// per cell) at the copy bandwidth, plus a launch.  TILED / TMA: per launch of
// up to 8 steps, the 128 x 80 region of T and P in and the 112 x 64 centre
// out (~15.4 bytes per output cell), and 8 steps of shared-memory work (~9
// bytes of shared traffic per cell and step, 1.43x redundant halo cells) at
// 128 bytes / clock / SM.
double stencil_prior_ms(int v, int64_t rows, int64_t cols, int iters, int num_sms) {
  const double cells = static_cast<double>(rows) * cols;
  const double bw = 6.4e12, smem = num_sms * 128.0 * 1.8e9;
  if (iters == 0) return 1e3 * cells * 8 / bw + 3e-3;
  if (v == COMPAR_S_NAIVE) return iters * (1e3 * cells * 12 / bw + 3e-3);
  const int launches = (iters + 7) / 8;
  const double per_launch = 1e3 * std::max(cells * 15.4 / bw, cells * 8 * 1.43 * 9 / smem);
  return launches * (per_launch * (v == COMPAR_S_TMA ? 0.95 : 1.0) + 4e-3);
}

int choose(compar_ctx* ctx, int64_t rows, int64_t cols, int iters, bool a16) {
  StencilSel& st = ctx->stencil;
  if (st.forced >= 0) return stencil_supported(st.forced, rows, cols, a16) ? st.forced
                                                                            : COMPAR_ERR_UNSUPPORTED;
  const auto key = std::make_tuple(rows, cols, iters);
  auto it = st.decisions.find(key);
  if (it != st.decisions.end() && stencil_supported(it->second, rows, cols, a16)) return it->second;
  int best = -1;
  double best_t = INFINITY;
  for (int v = 0; v < COMPAR_S_COUNT; ++v) {
    if (!stencil_supported(v, rows, cols, a16)) continue;
    double t = st.hist.predict(v, 0, rows, cols, std::max(iters, 1), 1, nullptr);
    if (t < 0) t = stencil_prior_ms(v, rows, cols, iters, ctx->num_sms);
    if (t < best_t) {
      best_t = t;
      best = v;
    }
  }
  if (best < 0) return COMPAR_ERR_UNSUPPORTED;
  st.decisions[key] = best;
  return best;
}

int check_call(compar_ctx* ctx, int64_t rows, int64_t cols, int iters,
               const compar_stencil_params_t* prm, const float* T_in, const float* P,
               const float* T_out) {
  if (!ctx || rows < 0 || cols < 0 || iters < 0 || !params_ok(prm)) return COMPAR_ERR_INVALID;
  if (rows == 0 || cols == 0) return COMPAR_OK;
  if (!T_in || !P || !T_out) return COMPAR_ERR_INVALID;
  for (const void* p : {static_cast<const void*>(T_in), static_cast<const void*>(P),
                        static_cast<const void*>(T_out)})
    if (reinterpret_cast<uintptr_t>(p) % 4) return COMPAR_ERR_INVALID;
  const size_t bytes = static_cast<size_t>(rows) * cols * sizeof(float);
  if (overlaps(T_out, T_in, bytes) || overlaps(T_out, P, bytes)) return COMPAR_ERR_INVALID;
  return COMPAR_OK;
}

int run_variant(compar_ctx* ctx, int v, int64_t rows, int64_t cols, int iters,
                const compar_stencil_params_t& prm, const float* T_in, const float* P,
                float* T_out, cudaStream_t s) {
  const size_t bytes = static_cast<size_t>(rows) * cols * sizeof(float);
  float* tmp = nullptr;
  if (iters > 1) {  // more than one launch: ping-pong through a scratch grid
    const int rc = ctx->ws.ensure((bytes + 255) / 256 * 256, s);
    if (rc != COMPAR_OK) return rc;
    tmp = static_cast<float*>(ctx->ws.ptr);
  }
  return stencil_launch(v, rows, cols, iters, prm, T_in, P, T_out, tmp, ctx->guard, s);
}

}  // namespace
}  // namespace compar

using namespace compar;

extern "C" {

int compar_stencil(compar_ctx_t ctx, int64_t rows, int64_t cols, int iters,
                   const compar_stencil_params_t* params, const float* T_in, const float* P,
                   float* T_out, void* stream) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  int rc = check_call(ctx, rows, cols, iters, params, T_in, P, T_out);
  if (rc != COMPAR_OK) return rc;
  if (ctx->host_only) return COMPAR_ERR_UNSUPPORTED;
  if (rows == 0 || cols == 0) return COMPAR_OK;
  const bool a16 = aligned16(T_in) && aligned16(P) && aligned16(T_out);
  const int v = choose(ctx, rows, cols, iters, a16);
  if (v < 0) return v;
  ctx->stencil.last = v;
  return run_variant(ctx, v, rows, cols, iters, *params, T_in, P, T_out,
                     static_cast<cudaStream_t>(stream));
}

int compar_stencil_force_variant(compar_ctx_t ctx, int v) {
  if (!ctx || v < -1 || v >= COMPAR_S_COUNT) return COMPAR_ERR_INVALID;
  ctx->stencil.forced = v;
  return COMPAR_OK;
}

int compar_stencil_last_variant(compar_ctx_t ctx) { return ctx ? ctx->stencil.last : -1; }

const char* compar_stencil_variant_name(int v) {
  return (v >= 0 && v < COMPAR_S_COUNT) ? kStencilNames[v] : nullptr;
}

int compar_stencil_supported(compar_ctx_t ctx, int v, int64_t rows, int64_t cols) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  if (!ctx || v < 0 || v >= COMPAR_S_COUNT || rows < 0 || cols < 0) return COMPAR_ERR_INVALID;
  if (v == COMPAR_S_TMA && ctx->host_only) return (cols % 4 == 0) ? 1 : 0;
  return stencil_supported(v, rows, cols, true) ? 1 : 0;
}

int compar_stencil_select(compar_ctx_t ctx, int64_t rows, int64_t cols, int iters) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  if (!ctx || rows <= 0 || cols <= 0 || iters < 0) return COMPAR_ERR_INVALID;
  if (ctx->host_only) {
    // no device to ask about TMA: decide by the grid alone
    StencilSel& st = ctx->stencil;
    if (st.forced >= 0) return st.forced;
    int best = -1;
    double best_t = INFINITY;
    for (int v = 0; v < COMPAR_S_COUNT; ++v) {
      if (v == COMPAR_S_TMA && cols % 4 != 0) continue;
      double t = st.hist.predict(v, 0, rows, cols, std::max(iters, 1), 1, nullptr);
      if (t < 0) t = stencil_prior_ms(v, rows, cols, iters, ctx->num_sms);
      if (t < best_t) {
        best_t = t;
        best = v;
      }
    }
    return best;
  }
  return choose(ctx, rows, cols, iters, true);
}

int compar_stencil_measure(compar_ctx_t ctx, int v, int64_t rows, int64_t cols, int iters,
                           const compar_stencil_params_t* params, const float* T_in,
                           const float* P, float* T_out, int warmup, int reps, void* stream,
                           float* median_ms) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  int rc = check_call(ctx, rows, cols, iters, params, T_in, P, T_out);
  if (rc != COMPAR_OK) return rc;
  if (v < 0 || v >= COMPAR_S_COUNT || reps < 1 || warmup < 0 || !median_ms || rows == 0 ||
      cols == 0)
    return COMPAR_ERR_INVALID;
  if (ctx->host_only) return COMPAR_ERR_UNSUPPORTED;
  rc = refuse_capture(static_cast<cudaStream_t>(stream), "compar_stencil_measure");
  if (rc != COMPAR_OK) return rc;  // it synchronises
  const bool a16 = aligned16(T_in) && aligned16(P) && aligned16(T_out);
  if (!stencil_supported(v, rows, cols, a16)) return COMPAR_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < warmup; ++i) {
    rc = run_variant(ctx, v, rows, cols, iters, *params, T_in, P, T_out, s);
    if (rc != COMPAR_OK) return rc;
  }
  rc = compar_check_device_error(ctx, s);
  if (rc != COMPAR_OK) return rc;
  std::vector<cudaEvent_t> ev(2 * reps);
  for (auto& e : ev) COMPAR_CUDA_TRY(cudaEventCreate(&e));
  for (int i = 0; i < reps && rc == COMPAR_OK; ++i) {
    cudaEventRecord(ev[2 * i], s);
    rc = run_variant(ctx, v, rows, cols, iters, *params, T_in, P, T_out, s);
    cudaEventRecord(ev[2 * i + 1], s);
  }
  std::vector<float> t;
  if (rc == COMPAR_OK && cudaEventSynchronize(ev.back()) != cudaSuccess) rc = COMPAR_ERR_CUDA;
  for (int i = 0; rc == COMPAR_OK && i < reps; ++i) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]) != cudaSuccess) rc = COMPAR_ERR_CUDA;
    t.push_back(ms);
  }
  for (auto e : ev) cudaEventDestroy(e);
  if (rc == COMPAR_OK) rc = compar_check_device_error(ctx, s);
  if (rc != COMPAR_OK) return rc;
  std::sort(t.begin(), t.end());
  const float med = (reps % 2) ? t[reps / 2] : 0.5f * (t[reps / 2 - 1] + t[reps / 2]);
  *median_ms = med;
  ctx->stencil.hist.observe(v, 0, rows, cols, std::max(iters, 1), 1, med);
  ctx->stencil.decisions.clear();
  return COMPAR_OK;
}

}  // extern "C"
