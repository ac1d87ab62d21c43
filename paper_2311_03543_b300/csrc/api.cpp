// The C ABI (include/compar.h): lifecycle, per-call variant selection and
// dispatch, forced variants, timing, records, selector files.
//
// Selection order for one call (Sec. 2.2: a task is mapped to one codelet of
// its set at run time; Sec. 3.2: the environment can pin the choice):
//   forced variant > decision cache > MLP cost model (when confident)
//   > history table > roofline prior,
// always restricted to the variants that can run the call and whose error
// model meets the tolerance.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <mutex>
#include <set>
#include <string>
#include <tuple>

#include "runtime.h"

namespace compar {

// ------------------------------------------------------------- errors
static thread_local std::string g_last_error;

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  g_last_error = buf;
}
std::string last_error_text() { return g_last_error; }
void set_last_error_text(const std::string& text) { g_last_error = text; }

int current_device_index() {
  int d = -1;
  if (cudaGetDevice(&d) != cudaSuccess) {
    (void)cudaGetLastError();
    return -1;
  }
  return (d >= 0 && d < kMaxDevices) ? d : -1;
}

cudaError_t smem_opt_in(const void* func, int bytes) {
  static std::mutex mu;
  static std::set<std::tuple<int, const void*, int>> done;
  const int d = current_device_index();
  if (d < 0) return cudaErrorInvalidDevice;
  const auto key = std::make_tuple(d, func, bytes);
  std::lock_guard<std::mutex> lock(mu);
  if (done.count(key)) return cudaSuccess;
  const cudaError_t e =
      cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.insert(key);
  return e;
}

DeviceScope::DeviceScope(int device) {
  if (device < 0) return;
  // A non-sticky error the caller left pending would otherwise be read by the
  // library's post-launch check as its own launch failing.
  (void)cudaGetLastError();
  if (cudaGetDevice(&prev_) != cudaSuccess) {
    (void)cudaGetLastError();
    return;
  }
  if (prev_ != device && cudaSetDevice(device) == cudaSuccess) switched_ = true;
}

DeviceScope::~DeviceScope() {
  if (switched_) cudaSetDevice(prev_);
}

// Growing a workspace inside a stream capture would hand the context memory
// that only the captured graph owns: refused (a call of the same shape before
// the capture grows it).
// Set when a call failed for a reason of the caller's (a workspace that
// would have to grow inside a stream capture, or device memory that ran
// out), not because its variant cannot run: such a failure is returned to
// the caller and quarantines nothing.
static thread_local bool g_transient_failure = false;

static int refuse_growth_in_capture(cudaStream_t s) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  COMPAR_CUDA_TRY(cudaStreamIsCapturing(s, &cap));
  if (cap == cudaStreamCaptureStatusNone) return COMPAR_OK;
  g_last_error =
      "the workspace must grow while the stream is captured: run the call once before capturing";
  g_transient_failure = true;
  return COMPAR_ERR_UNSUPPORTED;
}

int refuse_capture(cudaStream_t s, const char* call) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  COMPAR_CUDA_TRY(cudaStreamIsCapturing(s, &cap));
  if (cap == cudaStreamCaptureStatusNone) return COMPAR_OK;
  g_last_error = std::string(call) + " cannot be captured into a CUDA graph";
  return COMPAR_ERR_UNSUPPORTED;
}

static int workspace_alloc(void** p, size_t bytes, cudaStream_t s) {
  const cudaError_t e = cudaMallocAsync(p, bytes, s);
  if (e == cudaSuccess) return COMPAR_OK;
  (void)cudaGetLastError();
  *p = nullptr;
  set_last_cuda_error(e, "cudaMallocAsync (workspace)", __FILE__, __LINE__);
  g_transient_failure = true;
  return COMPAR_ERR_CUDA;
}

int Workspace::ensure(size_t need, cudaStream_t s) {
  if (need <= bytes) return COMPAR_OK;
  if (int rc = refuse_growth_in_capture(s); rc != COMPAR_OK) return rc;
  size_t grow = std::max(need, bytes + bytes / 2);
  grow = (grow + (1 << 20) - 1) & ~static_cast<size_t>((1 << 20) - 1);
  if (ptr) COMPAR_CUDA_TRY(cudaFreeAsync(ptr, s));
  ptr = nullptr;
  bytes = 0;
  if (int rc = workspace_alloc(&ptr, grow, s); rc != COMPAR_OK) return rc;
  bytes = grow;
  return COMPAR_OK;
}

int Workspace::ensure_counters(size_t n, cudaStream_t s) {
  if (n <= counter_n) return COMPAR_OK;
  if (int rc = refuse_growth_in_capture(s); rc != COMPAR_OK) return rc;
  const size_t grow = std::max<size_t>(n, 4096);
  if (counters) COMPAR_CUDA_TRY(cudaFreeAsync(counters, s));
  counters = nullptr;
  counter_n = 0;
  if (int rc = workspace_alloc(reinterpret_cast<void**>(&counters), grow * sizeof(*counters), s);
      rc != COMPAR_OK)
    return rc;
  COMPAR_CUDA_TRY(cudaMemsetAsync(counters, 0, grow * sizeof(*counters), s));
  counter_n = grow;
  return COMPAR_OK;
}

int Workspace::take_counters(size_t n, cudaStream_t s, uint32_t* epoch) {
  int rc = ensure_counters(n, s);
  if (rc != COMPAR_OK) return rc;
  *epoch = next_epoch();
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  COMPAR_CUDA_TRY(cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone)
    COMPAR_CUDA_TRY(cudaMemsetAsync(counters, 0, n * sizeof(*counters), s));
  return COMPAR_OK;
}

void Workspace::release() {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  bytes = 0;
  if (counters) cudaFree(counters);
  counters = nullptr;
  counter_n = 0;
}

static const char* kVariantNames[] = {"naive-f32", "simt-f32", "tc-tf32",
                                      "tc-bf16",   "tc-fp8",   "split-3xbf16",
                                      "grouped",   "split-6xbf16", "split-3xtf32",
                                      "split-3xbf16-fused"};
static_assert(sizeof(kVariantNames) / sizeof(kVariantNames[0]) == COMPAR_V_COUNT,
              "one name per variant id");

static double default_tol(double tol) { return tol > 0 ? tol : 1e-5; }

static int tol_class(double tol) { return static_cast<int>(std::floor(2.0 * std::log10(tol))); }

bool variant_supported(const compar_ctx* ctx, int v, const GemmCall& c) {
  (void)ctx;
  if (c.m > INT32_MAX || c.n > INT32_MAX || c.k > INT32_MAX) return false;
  switch (v) {
    case COMPAR_V_NAIVE:
      // one thread per output with a K-long FMA chain: never competitive
      // beyond ~2^36 multiply-adds, so not offered there
      return (c.m + 15) / 16 <= 65535 &&
             static_cast<double>(c.m) * c.n * c.k <= 68719476736.0;
    case COMPAR_V_SIMT:
      return (c.m + 31) / 32 <= 65535;
    case COMPAR_V_TC_TF32:
    case COMPAR_V_TC_BF16:
    case COMPAR_V_TC_FP8:
    case COMPAR_V_SPLIT3:
    case COMPAR_V_SPLIT6:
    case COMPAR_V_SPLIT3_TF32:
    case COMPAR_V_SPLIT3_FUSED:
      return tc_supported(v, c);
    default:
      return false;
  }
}

static int launch_variant(compar_ctx* ctx, int v, const GemmCall& c, cudaStream_t s) {
  if (v == ctx->test_fail_variant) {
    g_last_error = "injected failure (COMPAR_TEST_FAIL_VARIANT)";
    return COMPAR_ERR_CUDA;
  }
  switch (v) {
    case COMPAR_V_NAIVE: return launch_naive(c, ctx->guard, s);
    case COMPAR_V_SIMT: return launch_simt(c, ctx->ws, ctx->guard, ctx->num_sms, s);
    case COMPAR_V_TC_TF32:
    case COMPAR_V_TC_BF16:
    case COMPAR_V_TC_FP8:
    case COMPAR_V_SPLIT3:
    case COMPAR_V_SPLIT6:
    case COMPAR_V_SPLIT3_TF32:
    case COMPAR_V_SPLIT3_FUSED: return launch_tc(v, c, ctx->ws, ctx->guard, ctx->num_sms, s);
    default: return COMPAR_ERR_UNSUPPORTED;
  }
}

// Eligible variants for a call: runnable, not quarantined, error model within tol.
static uint32_t eligible_mask(const compar_ctx* ctx, const GemmCall& c) {
  uint32_t mask = 0;
  for (int v = 0; v < kNumVariants; ++v) {
    if (ctx->quarantined[v] || !variant_supported(ctx, v, c)) continue;
    // SIMT's error follows its longest FMA chain (split K shortens it)
    const int64_t k_chain = v == COMPAR_V_SIMT ? simt_plan(c, ctx->num_sms).k_per : c.k;
    if (ctx->err.predict(v, c.dtype, k_chain) * ctx->err.margin > c.tol) continue;
    mask |= 1u << v;
  }
  return mask;
}

// MLP choice; returns -1 when the model is untrained or not confident.
// `pred_all` (optional) receives the predicted time (ms) of every eligible
// variant that passes the learned error head, +inf for the others.
static int mlp_choice(compar_ctx* ctx, const GemmCall& c, uint32_t mask, float* pred_ms,
                      double* pred_all = nullptr) {
  const MlpModel& mm = ctx->mlp;
  if (!mm.trained) return -1;
  auto x = make_features(c.m, c.n, c.k, c.dtype, c.tol, c.batch);
  for (int i = 0; i < kNumFeatures; ++i) {  // outside the training box -> not confident
    const float span = mm.feat_max[i] - mm.feat_min[i];
    if (x[i] < mm.feat_min[i] - mm.box_slack * span - 1e-6f ||
        x[i] > mm.feat_max[i] + mm.box_slack * span + 1e-6f)
      return -1;
  }
  float out[kEnsemble * kOutputs];
  if (mlp_predict(ctx, x.data(), 1, out) != COMPAR_OK) return -1;
  int best = -1;
  float best_t = INFINITY, best_std = 0;
  for (int v = 0; v < kNumVariants; ++v) {
    if (!(mask & (1u << v))) continue;
    float mean_t = 0, mean_e = 0;
    for (int e = 0; e < kEnsemble; ++e) {
      mean_t += out[e * kOutputs + v];
      mean_e += out[e * kOutputs + kNumVariants + v];
    }
    mean_t /= kEnsemble;
    mean_e /= kEnsemble;
    // learned error head: log10 of the predicted relative error
    if (std::pow(10.f, mean_e) * ctx->err.margin > c.tol) continue;
    float var = 0;
    for (int e = 0; e < kEnsemble; ++e) {
      const float d = out[e * kOutputs + v] - mean_t;
      var += d * d;
    }
    // the time head predicts log2(measured / roofline prior)
    const float log2_t = mean_t + static_cast<float>(std::log2(
                                      prior_time_ms(v, c.m, c.n, c.k, c.dtype, ctx->num_sms)));
    if (pred_all) pred_all[v] = std::exp2(static_cast<double>(log2_t));
    if (log2_t < best_t) {
      best_t = log2_t;
      best = v;
      best_std = std::sqrt(var / kEnsemble);
    }
  }
  if (best < 0 || best_std > mm.conf_std) return -1;
  if (pred_ms) *pred_ms = std::exp2(best_t);
  return best;
}

static int history_choice(const compar_ctx* ctx, const GemmCall& c, uint32_t mask,
                          double* pred_ms, double* pred_all = nullptr) {
  int best = -1;
  double best_t = INFINITY;
  for (int v = 0; v < kNumVariants; ++v) {
    if (!(mask & (1u << v))) continue;
    double t = ctx->hist.predict(v, c.dtype, c.m, c.n, c.k, c.batch, nullptr);
    if (t < 0) t = prior_time_ms(v, c.m, c.n, c.k, c.dtype, ctx->num_sms);
    if (pred_all) pred_all[v] = t;
    if (t < best_t) {
      best_t = t;
      best = v;
    }
  }
  if (pred_ms) *pred_ms = best_t;
  return best;
}

// Chooses a variant; returns it or a negative status.
static int select_variant(compar_ctx* ctx, const GemmCall& c) {
  const uint32_t mask = eligible_mask(ctx, c);
  if (!mask) return COMPAR_ERR_NO_VARIANT;
  const DecisionKey key{c.m, c.n, c.k, static_cast<int>(c.dtype), tol_class(c.tol), c.batch};
  // Online exploration is drawn for every call, cached decision or not
  // (epsilon-greedy): a program that repeats its shapes keeps trying the
  // alternatives of its cached picks.
  auto next = [&]() {
    uint64_t z = (ctx->online.rng += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  const bool explore =
      ctx->online.epsilon > 0 &&
      static_cast<double>(next() >> 11) * (1.0 / 9007199254740992.0) < ctx->online.epsilon;
  auto it = ctx->decisions.find(key);
  const int cached =
      it != ctx->decisions.end() && (mask & (1u << it->second)) ? it->second : -1;
  if (cached >= 0 && !explore) return cached;
  int v = -1;
  const char* by = "history";
  float mlp_ms = 0;
  double hist_ms = 0;
  double pred[kNumVariants];
  for (double& t : pred) t = INFINITY;
  if (ctx->selector_mode != 1) {
    v = mlp_choice(ctx, c, mask, &mlp_ms, pred);
    if (v >= 0) by = "mlp";
  }
  if (v < 0 && ctx->selector_mode == 2 && ctx->mlp.trained) {
    // MLP-only mode still needs an answer when the ensemble disagrees
    by = "history(fallback)";
  }
  if (v < 0) {
    for (double& t : pred) t = INFINITY;
    v = history_choice(ctx, c, mask, &hist_ms, pred);
  }
  if (ctx->selector_mode != 2) {
    // Measured beats predicted: a variant timed in this call's own history
    // bucket (sizes within ~9 %) is ranked by its fastest measurement instead
    // of the model's estimate, so live timings correct the choice for the
    // shapes a program repeats, as a calibrated history model does.
    bool measured = false;
    int vm = -1;
    double best = INFINITY;
    for (int u = 0; u < kNumVariants; ++u) {
      if (!(mask & (1u << u))) continue;
      const double t = ctx->hist.measured_min(u, c.dtype, c.m, c.n, c.k, c.batch);
      const double e = t > 0 ? t : pred[u];
      measured = measured || t > 0;
      if (e < best) {
        best = e;
        vm = u;
      }
    }
    if (measured && vm >= 0 && vm != v) {
      v = vm;
      by = "measured";
    }
  }
  if (cached >= 0) v = cached;  // exploring around a cached decision
  if (explore) {
    // Exploration: run, once and without caching, another eligible variant
    // whose predicted time is within 4x of the pick's (any other eligible
    // variant when none is), so its timing is recorded where a mis-ranking
    // is plausible: the close calls are what the models must learn to rank.
    int ids[kNumVariants], nids = 0;
    for (int u = 0; u < kNumVariants; ++u)
      if (u != v && (mask & (1u << u)) && pred[u] <= 4.0 * pred[v]) ids[nids++] = u;
    if (nids == 0)
      for (int u = 0; u < kNumVariants; ++u)
        if (u != v && (mask & (1u << u))) ids[nids++] = u;
    if (nids > 0) {
      ctx->online.explored += 1;
      return ids[next() % static_cast<uint64_t>(nids)];
    }
    if (cached >= 0) return cached;
  }
  if (ctx->log)
    fprintf(stderr, "[compar] m=%lld n=%lld k=%lld dtype=%d tol=%.1e eligible=0x%x -> %s by %s\n",
            static_cast<long long>(c.m), static_cast<long long>(c.n),
            static_cast<long long>(c.k), static_cast<int>(c.dtype), c.tol, mask,
            kVariantNames[v], by);
  ctx->decisions[key] = v;
  return v;
}

static cudaEvent_t take_event(compar_ctx* ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    (void)cudaGetLastError();  // the call goes untimed
    return nullptr;
  }
  return e;
}

static void resolve_pending(compar_ctx* ctx) {
  for (auto& p : ctx->pending) {
    float ms = -1;
    if (cudaEventSynchronize(p.stop) == cudaSuccess &&
        cudaEventElapsedTime(&ms, p.start, p.stop) == cudaSuccess) {
      p.rec.time_ms = ms;
      ctx->rec.push(p.rec);
      ctx->hist.observe(p.rec.variant, p.rec.dtype, p.rec.m, p.rec.n, p.rec.k, p.rec.batch, ms);
    } else {
      (void)cudaGetLastError();  // a record lost, not an error of a later launch
    }
    ctx->event_pool.push_back(p.start);
    ctx->event_pool.push_back(p.stop);
  }
  ctx->pending.clear();
}

static compar_record_t make_record(const GemmCall& c, int v) {
  compar_record_t r{};
  r.m = c.m;
  r.n = c.n;
  r.k = c.k;
  r.dtype = c.dtype;
  r.variant = v;
  r.batch = c.batch;
  r.tol = static_cast<float>(c.tol);
  r.time_ms = -1;
  r.rel_err = -1;
  return r;
}

// The recorded-call gate's host-mapped word (allocated on first use); false
// when it cannot be had (the call is then timed without the gate).
static bool gate_ready(compar_ctx* ctx) {
  if (ctx->gate_dev) return true;
  void* h = nullptr;
  if (cudaHostAlloc(&h, sizeof(unsigned int), cudaHostAllocMapped) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  void* d = nullptr;
  if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
    (void)cudaGetLastError();
    cudaFreeHost(h);
    return false;
  }
  ctx->gate_host = static_cast<unsigned int*>(h);
  *ctx->gate_host = 0;
  ctx->gate_dev = static_cast<unsigned int*>(d);
  return true;
}

// Runs one call on variant v (recording it when recording is on).  A
// recorded call is held behind the gate kernel until all its launches are
// enqueued, so its recorded time is the device time of its kernels run back
// to back (as compar_measure times them), not host launch gaps.
static int run_one(compar_ctx* ctx, int v, const GemmCall& c, cudaStream_t s) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool gated = false;
  // A call captured into a graph is not timed: its events would belong to
  // the graph, not to this call.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  bool record = false;
  if (ctx->rec.on) {
    if (cudaStreamIsCapturing(s, &cap) == cudaSuccess) record = cap == cudaStreamCaptureStatusNone;
    else (void)cudaGetLastError();
  }
  if (record) {
    e0 = take_event(ctx);
    e1 = take_event(ctx);
    if (!e0 || !e1) {  // untimed: give back the one that was taken
      if (e0) ctx->event_pool.push_back(e0);
      if (e1) ctx->event_pool.push_back(e1);
      e0 = e1 = nullptr;
      record = false;
    }
    if (record && gate_ready(ctx))
      gated = launch_record_gate(ctx->gate_dev, ctx->gate_ticket + 1, s) == COMPAR_OK;
    if (e0) cudaEventRecord(e0, s);
  }
  const int rc = launch_variant(ctx, v, c, s);
  if (record && e0 && e1) cudaEventRecord(e1, s);
  if (gated) {
    // the whole call and its end event are enqueued: open the gate
    __atomic_store_n(ctx->gate_host, ++ctx->gate_ticket, __ATOMIC_RELEASE);
  }
  if (record && e0 && e1) {
    if (rc == COMPAR_OK) {
      ctx->pending.push_back(PendingTiming{e0, e1, make_record(c, v)});
      if (ctx->pending.size() >= 4096) resolve_pending(ctx);
    } else {
      ctx->event_pool.push_back(e0);
      ctx->event_pool.push_back(e1);
    }
  }
  return rc;
}

// Online mode: after `retrain_every` new timing records, fine-tune the MLP
// from its current weights on every record (synchronous, on the model's own
// stream) and start using it for new decisions.
static void maybe_retrain(compar_ctx* ctx, cudaStream_t s) {
  auto& o = ctx->online;
  if (o.retrain_every <= 0) return;
  const int64_t have = static_cast<int64_t>(ctx->rec.ring.size() + ctx->pending.size());
  if (have - o.records_at_train < o.retrain_every) return;
  // not while the caller's stream is captured: training synchronises
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    (void)cudaGetLastError();
    return;
  }
  if (cap != cudaStreamCaptureStatusNone) return;
  resolve_pending(ctx);
  const int steps = o.finetune_steps > 0 ? o.finetune_steps : 500;
  float vl = 0;
  const int rc = compar_selector_finetune(ctx, steps, 128, 5e-4f, 0xC0FFEEull + o.retrains, &vl);
  o.records_at_train = static_cast<int64_t>(ctx->rec.ring.size());
  if (ctx->log) fprintf(stderr, "[compar] online fine-tune rc=%d loss=%.4f\n", rc, vl);
}

int gemm_call(compar_ctx* ctx, GemmCall& c, cudaStream_t s) {
  if (c.m == 0 || c.n == 0) return COMPAR_OK;
  if (c.k == 0 || c.alpha == 0.f) {  // A and B are not read (BLAS convention)
    ctx->last_variant = -1;
    return launch_scale_c(c.C, c.m, c.n, c.ldc, c.beta, s);
  }
  if (ctx->forced >= 0) {
    if (!variant_supported(ctx, ctx->forced, c)) return COMPAR_ERR_UNSUPPORTED;
    ctx->last_variant = ctx->forced;
    return run_one(ctx, ctx->forced, c, s);
  }
  for (int attempt = 0; attempt < kNumVariants; ++attempt) {
    const int v = select_variant(ctx, c);
    if (v < 0) return v;
    ctx->last_variant = v;
    g_transient_failure = false;
    const int rc = run_one(ctx, v, c, s);
    if (rc == COMPAR_OK) {
      maybe_retrain(ctx, s);
      return rc;
    }
    if (g_transient_failure) return rc;  // the caller's condition: nothing quarantined
    // A variant that failed to launch is quarantined for this context and
    // the call is re-dispatched to the next choice.
    if (ctx->log)
      fprintf(stderr, "[compar] variant %s failed (%s); quarantined\n", kVariantNames[v],
              g_last_error.c_str());
    ctx->quarantined[v] = true;
    ctx->decisions.clear();
  }
  return COMPAR_ERR_NO_VARIANT;
}

static bool valid_dtype(int d) { return d == COMPAR_F32 || d == COMPAR_BF16 || d == COMPAR_F8E4M3; }

static int dtype_bytes_of(compar_dtype_t d) { return d == COMPAR_F32 ? 4 : (d == COMPAR_BF16 ? 2 : 1); }

// Contiguous operands of a call: C must not share a byte with A or B (a
// kernel would read what another writes).
static int check_ptrs(int64_t m, int64_t n, int64_t k, const void* A, const void* B,
                      const void* C, compar_dtype_t dtype) {
  if (m < 0 || n < 0 || k < 0) return COMPAR_ERR_INVALID;
  if (m > 0 && n > 0 && C == nullptr) return COMPAR_ERR_INVALID;
  if (m > 0 && n > 0 && k > 0 && (A == nullptr || B == nullptr)) return COMPAR_ERR_INVALID;
  if (C && (reinterpret_cast<uintptr_t>(C) % 4)) return COMPAR_ERR_INVALID;
  if (m > 0 && n > 0 && k > 0) {
    const uintptr_t c0 = reinterpret_cast<uintptr_t>(C);
    const uintptr_t c1 = c0 + static_cast<uintptr_t>(m) * n * 4;
    const uintptr_t e = static_cast<uintptr_t>(dtype_bytes_of(dtype));
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(A), a1 = a0 + static_cast<uintptr_t>(m) * k * e;
    const uintptr_t b0 = reinterpret_cast<uintptr_t>(B), b1 = b0 + static_cast<uintptr_t>(k) * n * e;
    if ((c0 < a1 && a0 < c1) || (c0 < b1 && b0 < c1)) {
      g_last_error = "C overlaps A or B";
      return COMPAR_ERR_INVALID;
    }
  }
  return COMPAR_OK;
}

}  // namespace compar

using namespace compar;

extern "C" {

int compar_init(compar_ctx_t* out, int device) {
  if (!out) return COMPAR_ERR_INVALID;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    (void)cudaGetLastError();
    g_last_error = "no such CUDA device";
    return COMPAR_ERR_CUDA;
  }
  cudaDeviceProp prop{};
  COMPAR_CUDA_TRY(cudaGetDeviceProperties(&prop, device));
  if (prop.major != 10 || prop.minor != 3) {
    g_last_error = "libcompar is built for sm_103 (B300) only";
    return COMPAR_ERR_UNSUPPORTED;
  }
  COMPAR_CUDA_TRY(cudaSetDevice(device));
  auto* ctx = new compar_ctx();
  ctx->device = device;
  ctx->guard.prof = &ctx->prof;
  ctx->num_sms = prop.multiProcessorCount;
  if (cudaMalloc(&ctx->guard.err_word, sizeof(int)) != cudaSuccess ||
      cudaMemset(ctx->guard.err_word, 0, sizeof(int)) != cudaSuccess) {
    g_last_error = "cannot allocate the device error word";
    delete ctx;
    return COMPAR_ERR_CUDA;
  }
  if (const char* e = getenv("COMPAR_FORCE_VARIANT")) ctx->forced = atoi(e);
  if (const char* e = getenv("COMPAR_SELECTOR")) {
    if (!strcmp(e, "history")) ctx->selector_mode = 1;
    else if (!strcmp(e, "mlp")) ctx->selector_mode = 2;
  }
  if (const char* e = getenv("COMPAR_LOG")) ctx->log = atoi(e) != 0;
  if (const char* e = getenv("COMPAR_WAIT_BUDGET_NS"))
    ctx->guard.budget_ns = std::max<unsigned long long>(1000, strtoull(e, nullptr, 10));
  if (const char* e = getenv("COMPAR_TEST_FAIL_VARIANT")) ctx->test_fail_variant = atoi(e);
  if (const char* e = getenv("COMPAR_SELECTOR_FILE")) {
    if (compar_selector_load(ctx, e) != COMPAR_OK && ctx->log)
      fprintf(stderr, "[compar] could not load selector file %s\n", e);
  }
  *out = ctx;
  return COMPAR_OK;
}

int compar_init_host(compar_ctx_t* out, int num_sms) {
  if (!out) return COMPAR_ERR_INVALID;
  auto* ctx = new compar_ctx();
  ctx->host_only = true;
  ctx->num_sms = num_sms > 0 ? num_sms : 148;
  ctx->device = -1;
  if (const char* e = getenv("COMPAR_LOG")) ctx->log = atoi(e) != 0;
  *out = ctx;
  return COMPAR_OK;
}

int compar_terminate(compar_ctx_t ctx) {
  if (!ctx) return COMPAR_OK;
  if (ctx->host_only) {
    delete ctx;
    return COMPAR_OK;
  }
  DeviceScope device_scope(ctx->device);
  cudaDeviceSynchronize();
  resolve_pending(ctx);
  for (auto e : ctx->event_pool) cudaEventDestroy(e);
  ctx->prof.release();
  batched_release(ctx);
  hostio_release(ctx);
  mlp_release(ctx);
  ctx->ws.release();
  if (ctx->gate_host) cudaFreeHost(ctx->gate_host);
  if (ctx->guard.err_word) cudaFree(ctx->guard.err_word);
  delete ctx;
  return COMPAR_OK;
}

const char* compar_status_string(int status) {
  switch (status) {
    case COMPAR_OK: return "ok";
    case COMPAR_ERR_INVALID: return "invalid argument";
    case COMPAR_ERR_UNSUPPORTED: return "unsupported";
    case COMPAR_ERR_CUDA: return "CUDA error";
    case COMPAR_ERR_TIMEOUT: return "device wait timed out";
    case COMPAR_ERR_IO: return "selector/record file error";
    case COMPAR_ERR_NO_VARIANT: return "no variant meets the tolerance";
    default: return "unknown status";
  }
}

const char* compar_last_error(void) { return g_last_error.c_str(); }

int compar_gemm(compar_ctx_t ctx, int64_t m, int64_t n, int64_t k, compar_dtype_t dtype,
                double tol, const void* A, const void* B, float* C, void* stream) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  if (!ctx || !valid_dtype(dtype) || std::isnan(tol)) return COMPAR_ERR_INVALID;
  if (ctx->host_only) return COMPAR_ERR_UNSUPPORTED;
  int rc = check_ptrs(m, n, k, A, B, C, dtype);
  if (rc != COMPAR_OK) return rc;
  GemmCall c;
  c.m = m;
  c.n = n;
  c.k = k;
  c.lda = k;
  c.ldb = n;
  c.ldc = n;
  c.dtype = dtype;
  c.tol = default_tol(tol);
  c.A = A;
  c.B = B;
  c.C = C;
  c.alpha = ctx->alpha;
  c.beta = ctx->beta;
  c.scale_a = ctx->scale_a;
  c.scale_b = ctx->scale_b;
  return gemm_call(ctx, c, static_cast<cudaStream_t>(stream));
}

int compar_gemm_host(compar_ctx_t ctx, int64_t m, int64_t n, int64_t k, compar_dtype_t dtype,
                     double tol, const void* A, const void* B, float* C, void* stream) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  if (!ctx || !valid_dtype(dtype) || std::isnan(tol)) return COMPAR_ERR_INVALID;
  if (ctx->host_only) return COMPAR_ERR_UNSUPPORTED;
  int rc = check_ptrs(m, n, k, A, B, C, dtype);
  if (rc != COMPAR_OK) return rc;
  // its copy streams and events are its own: not a capturable call
  rc = refuse_capture(static_cast<cudaStream_t>(stream), "compar_gemm_host");
  if (rc != COMPAR_OK) return rc;
  if (m == 0 || n == 0) return COMPAR_OK;
  GemmCall c;
  c.m = m;
  c.n = n;
  c.k = k;
  c.dtype = dtype;
  c.tol = default_tol(tol);
  c.alpha = ctx->alpha;
  c.beta = ctx->beta;
  c.scale_a = ctx->scale_a;
  c.scale_b = ctx->scale_b;
  return gemm_host(ctx, c, A, B, C, static_cast<cudaStream_t>(stream));
}

int compar_force_variant(compar_ctx_t ctx, int variant_id) {
  if (!ctx || variant_id < -1 || variant_id >= COMPAR_V_COUNT) return COMPAR_ERR_INVALID;
  ctx->forced = variant_id;
  return COMPAR_OK;
}

int compar_set_scalars(compar_ctx_t ctx, float alpha, float beta) {
  if (!ctx || !std::isfinite(alpha) || !std::isfinite(beta)) return COMPAR_ERR_INVALID;
  ctx->alpha = alpha;
  ctx->beta = beta;
  return COMPAR_OK;
}

int compar_set_fp8_scales(compar_ctx_t ctx, float scale_a, float scale_b) {
  if (!ctx || !(scale_a > 0) || !(scale_b > 0) || !std::isfinite(scale_a) ||
      !std::isfinite(scale_b))
    return COMPAR_ERR_INVALID;
  ctx->scale_a = scale_a;
  ctx->scale_b = scale_b;
  return COMPAR_OK;
}

int compar_set_selector_mode(compar_ctx_t ctx, int mode) {
  if (!ctx || mode < 0 || mode > 2) return COMPAR_ERR_INVALID;
  ctx->selector_mode = mode;
  ctx->decisions.clear();
  return COMPAR_OK;
}

int compar_last_variant(compar_ctx_t ctx) { return ctx ? ctx->last_variant : COMPAR_ERR_INVALID; }

int compar_variant_count(void) { return kNumVariants; }

const char* compar_variant_name(int v) {
  return (v >= 0 && v < COMPAR_V_COUNT) ? kVariantNames[v] : nullptr;
}

int compar_variant_supported(compar_ctx_t ctx, int v, int64_t m, int64_t n, int64_t k,
                             compar_dtype_t dtype) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  if (!ctx || v < 0 || v >= kNumVariants || !valid_dtype(dtype) || m < 0 || n < 0 || k < 0)
    return COMPAR_ERR_INVALID;
  GemmCall c;
  c.m = m;
  c.n = n;
  c.k = k;
  c.lda = k;  // contiguous operands
  c.ldb = n;
  c.ldc = n;
  c.dtype = dtype;
  return variant_supported(ctx, v, c) ? 1 : 0;
}

int compar_clear_decisions(compar_ctx_t ctx) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  if (!ctx) return COMPAR_ERR_INVALID;
  ctx->decisions.clear();
  return COMPAR_OK;
}

int compar_select(compar_ctx_t ctx, int64_t m, int64_t n, int64_t k, compar_dtype_t dtype,
                  double tol, int batch) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  if (!ctx || !valid_dtype(dtype) || std::isnan(tol) || m <= 0 || n <= 0 || k <= 0 ||
      batch < 1)
    return COMPAR_ERR_INVALID;
  GemmCall c;
  c.m = m;
  c.n = n;
  c.k = k;
  c.lda = k;
  c.ldb = n;
  c.ldc = n;
  c.dtype = dtype;
  c.tol = default_tol(tol);
  c.batch = batch;
  if (ctx->forced >= 0)
    return variant_supported(ctx, ctx->forced, c) ? ctx->forced : COMPAR_ERR_UNSUPPORTED;
  return select_variant(ctx, c);
}

int compar_error_model_set(compar_ctx_t ctx, int v, compar_dtype_t dtype, double c0, double c1,
                           double c2) {
  if (!ctx || v < 0 || v >= kNumVariants || !valid_dtype(dtype) || std::isnan(c0) ||
      !(c1 >= 0) || !(c2 >= 0) || !std::isfinite(c1) || !std::isfinite(c2) || c0 < 0)
    return COMPAR_ERR_INVALID;
  ctx->err.c0[v][dtype] = static_cast<float>(c0);
  ctx->err.c1[v][dtype] = static_cast<float>(c1);
  ctx->err.c2[v][dtype] = static_cast<float>(c2);
  ctx->decisions.clear();
  return COMPAR_OK;
}

int compar_error_model_get(compar_ctx_t ctx, int v, compar_dtype_t dtype, double* c0, double* c1,
                           double* c2) {
  if (!ctx || v < 0 || v >= kNumVariants || !valid_dtype(dtype) || !c0 || !c1 || !c2)
    return COMPAR_ERR_INVALID;
  *c0 = ctx->err.c0[v][dtype];
  *c1 = ctx->err.c1[v][dtype];
  *c2 = ctx->err.c2[v][dtype];
  return COMPAR_OK;
}

int compar_error_model_set_margin(compar_ctx_t ctx, double margin) {
  if (!ctx || !(margin >= 1.0) || !std::isfinite(margin)) return COMPAR_ERR_INVALID;
  ctx->err.margin = static_cast<float>(margin);
  ctx->decisions.clear();
  return COMPAR_OK;
}

double compar_error_model_predict(compar_ctx_t ctx, int v, compar_dtype_t dtype, int64_t k) {
  if (!ctx || v < 0 || v >= kNumVariants || !valid_dtype(dtype) || k < 0) return -1.0;
  return ctx->err.predict(v, dtype, k);
}

int compar_measure(compar_ctx_t ctx, int v, int64_t m, int64_t n, int64_t k,
                   compar_dtype_t dtype, double tol, const void* A, const void* B, float* C,
                   int warmup, int reps, void* stream, float* median_ms) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  if (!ctx || !median_ms || v < 0 || v >= kNumVariants || !valid_dtype(dtype) || reps < 1 ||
      warmup < 0)
    return COMPAR_ERR_INVALID;
  if (ctx->host_only) return COMPAR_ERR_UNSUPPORTED;
  int rc = check_ptrs(m, n, k, A, B, C, dtype);
  if (rc != COMPAR_OK) return rc;
  if (m == 0 || n == 0 || k == 0) return COMPAR_ERR_INVALID;
  rc = refuse_capture(static_cast<cudaStream_t>(stream), "compar_measure");  // it synchronises
  if (rc != COMPAR_OK) return rc;
  GemmCall c;
  c.m = m;
  c.n = n;
  c.k = k;
  c.lda = k;
  c.ldb = n;
  c.ldc = n;
  c.dtype = dtype;
  c.tol = default_tol(tol);
  c.A = A;
  c.B = B;
  c.C = C;
  c.alpha = ctx->alpha;
  c.beta = ctx->beta;
  c.scale_a = ctx->scale_a;
  c.scale_b = ctx->scale_b;
  if (!variant_supported(ctx, v, c)) return COMPAR_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < warmup; ++i) {
    rc = launch_variant(ctx, v, c, s);
    if (rc != COMPAR_OK) return rc;
  }
  // a kernel whose bounded wait ran out reports it here, before any timing
  rc = compar_check_device_error(ctx, s);
  if (rc != COMPAR_OK) return rc;
  std::vector<cudaEvent_t> ev(2 * reps);
  for (auto& e : ev) {
    e = take_event(ctx);
    if (!e) return COMPAR_ERR_CUDA;
  }
  for (int i = 0; i < reps; ++i) {
    cudaEventRecord(ev[2 * i], s);
    rc = launch_variant(ctx, v, c, s);
    cudaEventRecord(ev[2 * i + 1], s);
    if (rc != COMPAR_OK) break;
  }
  std::vector<float> t;
  if (rc == COMPAR_OK) {
    if (cudaEventSynchronize(ev.back()) != cudaSuccess) rc = COMPAR_ERR_CUDA;
    for (int i = 0; rc == COMPAR_OK && i < reps; ++i) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]) != cudaSuccess) {
        rc = COMPAR_ERR_CUDA;
        break;
      }
      t.push_back(ms);
    }
  }
  for (auto e : ev) ctx->event_pool.push_back(e);
  if (rc == COMPAR_OK) rc = compar_check_device_error(ctx, s);
  if (rc != COMPAR_OK) return rc;  // no timing of a failed run reaches the models
  if (ctx->rec.on) {
    for (float ms : t) {
      compar_record_t r = make_record(c, v);
      r.time_ms = ms;
      ctx->rec.push(r);
    }
  }
  std::sort(t.begin(), t.end());
  const float med = (reps % 2) ? t[reps / 2] : 0.5f * (t[reps / 2 - 1] + t[reps / 2]);
  *median_ms = med;
  ctx->hist.observe(v, dtype, m, n, k, 1, med);
  return COMPAR_OK;
}

int compar_record_enable(compar_ctx_t ctx, int on) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  if (!ctx) return COMPAR_ERR_INVALID;
  if (!on) resolve_pending(ctx);
  ctx->rec.on = on != 0;
  return COMPAR_OK;
}

int64_t compar_record_count(compar_ctx_t ctx) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  if (!ctx) return COMPAR_ERR_INVALID;
  resolve_pending(ctx);
  return static_cast<int64_t>(ctx->rec.ring.size());
}

int64_t compar_record_get(compar_ctx_t ctx, compar_record_t* out, int64_t max) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  if (!ctx || (!out && max > 0) || max < 0) return COMPAR_ERR_INVALID;
  resolve_pending(ctx);
  auto snap = ctx->rec.snapshot();
  const int64_t nout = std::min<int64_t>(max, static_cast<int64_t>(snap.size()));
  if (nout > 0) memcpy(out, snap.data(), static_cast<size_t>(nout) * sizeof(compar_record_t));
  return nout;
}

int compar_record_add(compar_ctx_t ctx, const compar_record_t* recs, int64_t count) {
  if (!ctx || count < 0 || (count > 0 && !recs)) return COMPAR_ERR_INVALID;
  for (int64_t i = 0; i < count; ++i) {
    const compar_record_t& r = recs[i];
    if (r.variant < 0 || r.variant >= kNumVariants || !valid_dtype(r.dtype)) return COMPAR_ERR_INVALID;
    ctx->rec.push(r);
    if (r.time_ms > 0) ctx->hist.observe(r.variant, r.dtype, r.m, r.n, r.k, r.batch, r.time_ms);
  }
  return COMPAR_OK;
}

int compar_record_clear(compar_ctx_t ctx) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  if (!ctx) return COMPAR_ERR_INVALID;
  resolve_pending(ctx);
  ctx->rec.clear();
  return COMPAR_OK;
}

int compar_check_device_error(compar_ctx_t ctx, void* stream) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  if (!ctx) return COMPAR_ERR_INVALID;
  if (ctx->host_only) return COMPAR_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int word = 0;
  COMPAR_CUDA_TRY(cudaMemcpyAsync(&word, ctx->guard.err_word, sizeof(int),
                                  cudaMemcpyDeviceToHost, s));
  COMPAR_CUDA_TRY(cudaMemsetAsync(ctx->guard.err_word, 0, sizeof(int), s));
  COMPAR_CUDA_TRY(cudaStreamSynchronize(s));
  return word == 0 ? COMPAR_OK : word;
}

int compar_set_wait_budget(compar_ctx_t ctx, uint64_t ns) {
  if (!ctx) return COMPAR_ERR_INVALID;
  ctx->guard.budget_ns = std::max<uint64_t>(ns, 1000);
  return COMPAR_OK;
}

int compar_selftest_timeout(compar_ctx_t ctx, void* stream) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  if (!ctx) return COMPAR_ERR_INVALID;
  if (ctx->host_only) return COMPAR_ERR_UNSUPPORTED;
  return launch_timeout_selftest(ctx->guard, static_cast<cudaStream_t>(stream));
}

int compar_tc_plan(int variant_id, int64_t m, int64_t n, int64_t k, int num_sms, int64_t* out) {
  return tc_plan_info(variant_id, m, n, k, num_sms, out, false);
}

int compar_tc_pair_plan(int variant_id, int64_t m, int64_t n, int64_t k, int num_pairs,
                        int64_t* out) {
  return tc_plan_info(variant_id, m, n, k, num_pairs, out, true);
}

int compar_set_tc_pairs(compar_ctx_t ctx, int mode) {
  if (!ctx || mode < -1 || mode > 1) return COMPAR_ERR_INVALID;
  ctx->guard.tc_pair = mode;
  return COMPAR_OK;
}

int compar_simt_plan(int64_t m, int64_t n, int64_t k, compar_dtype_t dtype, int64_t ldb,
                     int num_sms, int64_t* out) {
  if (!out || m < 1 || n < 1 || k < 1 || ldb < n || num_sms < 1 ||
      (dtype != COMPAR_F32 && dtype != COMPAR_BF16 && dtype != COMPAR_F8E4M3))
    return COMPAR_ERR_INVALID;
  GemmCall c;
  c.m = m;
  c.n = n;
  c.k = k;
  c.lda = k;
  c.ldb = ldb;
  c.ldc = n;
  c.dtype = dtype;
  const SimtPlan p = simt_plan(c, num_sms);
  out[0] = p.skinny ? 1 : 0;
  out[1] = p.bm;
  out[2] = p.bn;
  out[3] = p.splits;
  out[4] = p.k_per;
  out[5] = p.cluster;
  return COMPAR_OK;
}

}  // extern "C"
