// Host-side runtime of libcompar: the context, the variant registry with its
// eligibility rules and error model, the history-table and MLP cost models,
// the timing recorder and the decision cache.  Sec. 2.2 ("Runtime System")
// describes the paper's runtime (StarPU): a task has several codelets (one
// per implementation variant) and the runtime chooses one per task with
// performance models; this is that role for one GEMM component on one GPU.
#pragma once

#include <array>
#include <cstdint>
#include <cmath>
#include <map>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "common.h"

namespace compar {

constexpr int kNumVariants = COMPAR_V_COUNT;  // variant ids 0..8 (6: batched only)
constexpr int kNumFeatures = 8;
constexpr int kHidden = 64;
constexpr int kOutputs = 2 * kNumVariants;  // log time, log error per variant
constexpr int kEnsemble = 4;

// ------------------------------------------------------------- features
// x = (log2 M, log2 N, log2 K, [dtype==f32], [dtype==bf16], [dtype==f8],
//      log10 tol, log2 batch)
std::array<float, kNumFeatures> make_features(int64_t m, int64_t n, int64_t k, int dtype,
                                              double tol, int batch);

// ------------------------------------------------------------- error model
// Predicted relative Frobenius error of variant v on inputs of `dtype` with
// inner dimension k:  err = c0 + c1 * sqrt(k) * 2^-24.  Calibrated values can
// be loaded from a selector file.
struct ErrorModel {
  std::array<std::array<float, 3>, kNumVariants> c0{};
  std::array<std::array<float, 3>, kNumVariants> c1{};
  std::array<std::array<float, 3>, kNumVariants> c2{};  // linear-in-k term
  float margin = 1.25f;  // eligibility: predicted * margin <= tol
  ErrorModel();
  double predict(int v, int dtype, int64_t k) const;
};

// ------------------------------------------------------------- history table
// Key: (variant, dtype, round(4 log2 M), round(4 log2 N), round(4 log2 K),
// batch bucket) -> running mean of the measured time.  A miss takes the
// nearest key of the same variant and dtype (L1 distance in the quarter-log
// grid, at most kMaxDist) scaled by the ratio of 2MNK; with no such key the
// roofline prior answers.
struct HistKey {
  int8_t v, dtype;
  int16_t lm, ln, lk;
  int8_t batch;
  bool operator<(const HistKey& o) const;
  bool operator==(const HistKey& o) const;
};
struct HistVal {
  double mean_ms = 0;
  double m2 = 0;
  int64_t count = 0;
  // fastest observation: ranks measured variants (a cold first call or a
  // disturbed run does not decide against a variant)
  double min_ms = INFINITY;
};
struct HistoryModel {
  std::map<HistKey, HistVal> table;
  static constexpr int kMaxDist = 6;
  static HistKey key(int v, int dtype, int64_t m, int64_t n, int64_t k, int batch);
  void observe(int v, int dtype, int64_t m, int64_t n, int64_t k, int batch, double ms);
  // Predicted time in ms; *exact receives whether the key was present.
  // Returns < 0 when nothing near is known.
  double predict(int v, int dtype, int64_t m, int64_t n, int64_t k, int batch, bool* exact) const;
  // Fastest time observed in the call's own bucket, or < 0 if none.
  double measured_min(int v, int dtype, int64_t m, int64_t n, int64_t k, int batch) const;
};

// Roofline prior: max(work / pipe peak, bytes / bandwidth) + launch overheads.
double prior_time_ms(int v, int64_t m, int64_t n, int64_t k, int dtype, int num_sms);

// ------------------------------------------------------------- MLP model
struct MlpParams {  // one ensemble member, row-major (out, in)
  std::vector<float> W1, b1, W2, b2, W3, b3;
  void init(uint64_t seed);
  static size_t count();
  void flatten(std::vector<float>& out) const;
  void unflatten(const float* p);
};
struct MlpModel {
  bool trained = false;
  std::array<MlpParams, kEnsemble> members;
  std::array<float, kNumFeatures> feat_mean{}, feat_std{};
  std::array<float, kNumFeatures> feat_min{}, feat_max{};
  std::array<float, kOutputs> out_mean{}, out_std{};  // target standardisation
  float conf_std = 0.15f;  // max ensemble std of predicted log time
  float box_slack = 0.10f; // fraction of the training range allowed outside
};

// ------------------------------------------------------------- records
struct Recorder {
  bool on = false;
  std::vector<compar_record_t> ring;
  int64_t head = 0, size = 0;
  static constexpr int64_t kCap = 1 << 20;
  void push(const compar_record_t& r);
  std::vector<compar_record_t> snapshot() const;
  void clear() { head = size = 0; ring.clear(); }
};

struct DecisionKey {
  int64_t m, n, k;
  int dtype;
  int tol_class;
  int batch;
  bool operator==(const DecisionKey& o) const {
    return m == o.m && n == o.n && k == o.k && dtype == o.dtype && tol_class == o.tol_class &&
           batch == o.batch;
  }
};
struct DecisionKeyHash {
  size_t operator()(const DecisionKey& d) const;
};

// Selection state of the thermal-stencil component: forced variant, the
// variant of the last call, a history table keyed by (variant, rows, cols,
// iterations) and the decision cache.
struct StencilSel {
  int forced = -1;
  int last = -1;
  HistoryModel hist;
  std::map<std::tuple<int64_t, int64_t, int>, int> decisions;
};

struct PendingTiming {  // events of a recorded compar_gemm call, resolved lazily
  cudaEvent_t start, stop;
  compar_record_t rec;
};

}  // namespace compar

// The opaque context of the C ABI.
// Internal status of a warm fine-tune whose result was discarded (the
// model is unchanged); never returned through the C ABI.
constexpr int COMPAR_FINETUNE_KEPT = 1;

struct compar_ctx {
  bool host_only = false;  // created by compar_init_host: no CUDA calls at all
  int device = 0;
  int num_sms = 148;
  float alpha = 1.f, beta = 0.f;
  float scale_a = 1.f, scale_b = 1.f;
  int forced = -1;
  int selector_mode = 0;  // 0 auto, 1 history, 2 mlp
  int last_variant = -1;
  bool log = false;
  int test_fail_variant = -1;                 // host-side fault injection
  std::array<bool, compar::kNumVariants> quarantined{};
  compar::Workspace ws;
  compar::DeviceGuard guard;
  compar::KernelProfiler prof;
  compar::ErrorModel err;
  compar::HistoryModel hist;
  compar::MlpModel mlp;
  compar::Recorder rec;
  // A sample of the timing records the loaded MLP was trained on (from the
  // selector file): online fine-tunes train on it together with the live
  // records, so that they add what is new instead of forgetting the rest.
  std::vector<compar_record_t> rehearsal;
  std::unordered_map<compar::DecisionKey, int, compar::DecisionKeyHash> decisions;
  std::vector<compar::PendingTiming> pending;
  std::vector<cudaEvent_t> event_pool;
  // batch signature -> autotuned batched configuration (0 loop, 1..4 grouped)
  std::unordered_map<uint64_t, int> batched_cfg;
  int batched_forced = -1;  // compar_set_batched_config
  // online selection: exploration probability on decision-cache misses and
  // warm-start fine-tuning of the MLP every `retrain_every` new records
  struct Online {
    double epsilon = 0.0;
    int64_t retrain_every = 0;
    int finetune_steps = 0;
    int64_t records_at_train = 0;
    uint64_t rng = 0x243F6A8885A308D3ull;
    int64_t explored = 0, retrains = 0, rejected = 0;
  } online;
  void* batched_state = nullptr;
  void* hostio_state = nullptr;  // device buffers and streams of compar_gemm_host
  compar::StencilSel stencil;    // the second component's selection state
  // MLP device buffers (selector inference / training), owned here.
  void* mlp_dev = nullptr;
  // recorded-call gate: a host-mapped word and the last ticket written
  unsigned int* gate_host = nullptr;
  unsigned int* gate_dev = nullptr;
  unsigned int gate_ticket = 0;
};

namespace compar {
// Implemented in selector_mlp.cpp / mlp.cu
int mlp_predict(compar_ctx* ctx, const float* feats, int rows, float* out_host);
void mlp_release(compar_ctx* ctx);
// Implemented in batched.cpp
void batched_release(compar_ctx* ctx);
// Implemented in hostio.cpp
int gemm_host(compar_ctx* ctx, GemmCall base, const void* hA, const void* hB, float* hC,
              cudaStream_t s);
void hostio_release(compar_ctx* ctx);
}  // namespace compar
