// Host side of the learned cost model: feature / target standardisation,
// training-set assembly from the context's timing records, the ensemble's
// device buffers, inference for selection, and the C-ABI entry points of the
// MLP kernels (mlp.cu).
//
// Training (compar_selector_train): each record becomes one row; its time
// (log2 ms) and, when measured, its relative error (log10) are the targets of
// its variant's two outputs, every other output is masked.  The tolerance
// feature is drawn at random from {1e-5, 1e-3, 1e-1} for every row (time and
// error do not depend on the tolerance asked, so the model learns to ignore
// it).  Each of the 4 ensemble members trains on its own bootstrap sample of
// mini-batches; the spread of their predictions is the confidence signal.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "runtime.h"

namespace compar {

int mlp_param_count();
int mlp_forward_device(const float* d_params, int members, const float* d_X, int rows,
                       float* d_Y, cudaStream_t s);
int mlp_train_device(float* d_params, float* d_m, float* d_v, int members, const float* d_X,
                     const float* d_T, const float* d_M, const int* d_idx, int steps, int batch,
                     float lr, int step0, int apply, float* d_grads, float* d_loss,
                     cudaStream_t s);

namespace {

struct MlpDevice {
  cudaStream_t stream = nullptr;
  float* params = nullptr;  // [kEnsemble][P] of the trained model
  bool uploaded = false;
  float* x = nullptr;       // inference staging
  float* y = nullptr;
  int cap_rows = 0;
};

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

MlpDevice* dev_state(compar_ctx* ctx) {
  if (!ctx->mlp_dev) {
    auto* d = new MlpDevice();
    if (cudaStreamCreateWithFlags(&d->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete d;
      return nullptr;
    }
    ctx->mlp_dev = d;
  }
  return static_cast<MlpDevice*>(ctx->mlp_dev);
}

template <typename T>
int dev_alloc(T** p, size_t count) {
  COMPAR_CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T)));
  return COMPAR_OK;
}

// RAII list of device buffers for one training call.
struct Buffers {
  std::vector<void*> ptrs;
  template <typename T>
  int get(T** p, size_t count) {
    int rc = dev_alloc(p, count);
    if (rc == COMPAR_OK) ptrs.push_back(*p);
    return rc;
  }
  ~Buffers() {
    for (void* p : ptrs) cudaFree(p);
  }
};

int upload_model(compar_ctx* ctx, MlpDevice* d) {
  const size_t P = MlpParams::count();
  if (!d->params) {
    int rc = dev_alloc(&d->params, kEnsemble * P);
    if (rc != COMPAR_OK) return rc;
  }
  std::vector<float> flat, all;
  for (const auto& m : ctx->mlp.members) {
    m.flatten(flat);
    all.insert(all.end(), flat.begin(), flat.end());
  }
  COMPAR_CUDA_TRY(cudaMemcpy(d->params, all.data(), all.size() * sizeof(float),
                             cudaMemcpyHostToDevice));
  d->uploaded = true;
  return COMPAR_OK;
}

}  // namespace

void mlp_release(compar_ctx* ctx) {
  auto* d = static_cast<MlpDevice*>(ctx->mlp_dev);
  if (!d) return;
  if (d->stream) cudaStreamSynchronize(d->stream);
  cudaFree(d->params);
  cudaFree(d->x);
  cudaFree(d->y);
  if (d->stream) cudaStreamDestroy(d->stream);
  delete d;
  ctx->mlp_dev = nullptr;
}

// Raw features of `rows` contexts -> de-standardised outputs of every member:
// out_host[(e * rows + r) * kOutputs + o] (log2 ms, log10 error).
int mlp_predict(compar_ctx* ctx, const float* feats, int rows, float* out_host) {
  if (ctx->host_only || !ctx->mlp.trained) return COMPAR_ERR_UNSUPPORTED;
  MlpDevice* d = dev_state(ctx);
  if (!d) return COMPAR_ERR_CUDA;
  if (!d->uploaded) {
    int rc = upload_model(ctx, d);
    if (rc != COMPAR_OK) return rc;
  }
  if (rows > d->cap_rows) {
    cudaFree(d->x);
    cudaFree(d->y);
    d->x = d->y = nullptr;
    d->cap_rows = 0;
    int rc = dev_alloc(&d->x, static_cast<size_t>(rows) * kNumFeatures);
    if (rc == COMPAR_OK) rc = dev_alloc(&d->y, static_cast<size_t>(rows) * kEnsemble * kOutputs);
    if (rc != COMPAR_OK) return rc;
    d->cap_rows = rows;
  }
  const MlpModel& mm = ctx->mlp;
  std::vector<float> x(static_cast<size_t>(rows) * kNumFeatures);
  for (int r = 0; r < rows; ++r)
    for (int j = 0; j < kNumFeatures; ++j)
      x[r * kNumFeatures + j] = (feats[r * kNumFeatures + j] - mm.feat_mean[j]) / mm.feat_std[j];
  COMPAR_CUDA_TRY(cudaMemcpyAsync(d->x, x.data(), x.size() * sizeof(float),
                                  cudaMemcpyHostToDevice, d->stream));
  int rc = mlp_forward_device(d->params, kEnsemble, d->x, rows, d->y, d->stream);
  if (rc != COMPAR_OK) return rc;
  const size_t ny = static_cast<size_t>(rows) * kEnsemble * kOutputs;
  COMPAR_CUDA_TRY(cudaMemcpyAsync(out_host, d->y, ny * sizeof(float), cudaMemcpyDeviceToHost,
                                  d->stream));
  COMPAR_CUDA_TRY(cudaStreamSynchronize(d->stream));
  for (size_t i = 0; i < ny; ++i) {
    const int o = static_cast<int>(i % kOutputs);
    out_host[i] = out_host[i] * mm.out_std[o] + mm.out_mean[o];
  }
  return COMPAR_OK;
}

}  // namespace compar

using namespace compar;

extern "C" {

int compar_mlp_param_count(void) { return mlp_param_count(); }

int compar_mlp_forward(compar_ctx_t ctx, const float* params, int members, const float* X,
                       int rows, float* Y) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  if (!ctx || !params || !X || !Y || members <= 0 || rows <= 0) return COMPAR_ERR_INVALID;
  if (ctx->host_only) return COMPAR_ERR_UNSUPPORTED;
  MlpDevice* d = dev_state(ctx);
  if (!d) return COMPAR_ERR_CUDA;
  const size_t P = MlpParams::count();
  Buffers b;
  float *dp, *dx, *dy;
  int rc = b.get(&dp, members * P);
  if (rc == COMPAR_OK) rc = b.get(&dx, static_cast<size_t>(rows) * kNumFeatures);
  if (rc == COMPAR_OK) rc = b.get(&dy, static_cast<size_t>(rows) * members * kOutputs);
  if (rc != COMPAR_OK) return rc;
  COMPAR_CUDA_TRY(cudaMemcpyAsync(dp, params, members * P * sizeof(float), cudaMemcpyHostToDevice,
                                  d->stream));
  COMPAR_CUDA_TRY(cudaMemcpyAsync(dx, X, static_cast<size_t>(rows) * kNumFeatures * sizeof(float),
                                  cudaMemcpyHostToDevice, d->stream));
  rc = mlp_forward_device(dp, members, dx, rows, dy, d->stream);
  if (rc != COMPAR_OK) return rc;
  COMPAR_CUDA_TRY(cudaMemcpyAsync(Y, dy,
                                  static_cast<size_t>(rows) * members * kOutputs * sizeof(float),
                                  cudaMemcpyDeviceToHost, d->stream));
  COMPAR_CUDA_TRY(cudaStreamSynchronize(d->stream));
  return COMPAR_OK;
}

int compar_mlp_train_steps(compar_ctx_t ctx, float* params, float* adam_m, float* adam_v,
                           int members, const float* X, const float* T, const float* mask,
                           int rows, const int32_t* batch_idx, int steps, int batch, float lr,
                           int step0, float* grads, float* loss) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  if (!ctx || !params || !X || !T || !mask || !batch_idx || members <= 0 || rows <= 0 ||
      steps <= 0 || batch <= 0 || batch > 128 || step0 < 1 || !(lr >= 0))
    return COMPAR_ERR_INVALID;
  if (!grads && (!adam_m || !adam_v)) return COMPAR_ERR_INVALID;
  if (grads && steps != 1) return COMPAR_ERR_INVALID;
  for (int64_t i = 0; i < static_cast<int64_t>(members) * steps * batch; ++i)
    if (batch_idx[i] < 0 || batch_idx[i] >= rows) return COMPAR_ERR_INVALID;
  if (ctx->host_only) return COMPAR_ERR_UNSUPPORTED;
  MlpDevice* d = dev_state(ctx);
  if (!d) return COMPAR_ERR_CUDA;
  const size_t P = MlpParams::count();
  Buffers b;
  float *dp, *dm, *dv, *dx, *dt, *dmask, *dg = nullptr, *dl;
  int* di;
  int rc = b.get(&dp, members * P);
  if (rc == COMPAR_OK) rc = b.get(&dm, members * P);
  if (rc == COMPAR_OK) rc = b.get(&dv, members * P);
  if (rc == COMPAR_OK) rc = b.get(&dx, static_cast<size_t>(rows) * kNumFeatures);
  if (rc == COMPAR_OK) rc = b.get(&dt, static_cast<size_t>(rows) * kOutputs);
  if (rc == COMPAR_OK) rc = b.get(&dmask, static_cast<size_t>(rows) * kOutputs);
  if (rc == COMPAR_OK) rc = b.get(&di, static_cast<size_t>(members) * steps * batch);
  if (rc == COMPAR_OK) rc = b.get(&dl, static_cast<size_t>(members) * steps);
  if (rc == COMPAR_OK && grads) rc = b.get(&dg, members * P);
  if (rc != COMPAR_OK) return rc;
  auto h2d = [&](void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, d->stream);
  };
  COMPAR_CUDA_TRY(h2d(dp, params, members * P * sizeof(float)));
  if (adam_m) COMPAR_CUDA_TRY(h2d(dm, adam_m, members * P * sizeof(float)));
  else COMPAR_CUDA_TRY(cudaMemsetAsync(dm, 0, members * P * sizeof(float), d->stream));
  if (adam_v) COMPAR_CUDA_TRY(h2d(dv, adam_v, members * P * sizeof(float)));
  else COMPAR_CUDA_TRY(cudaMemsetAsync(dv, 0, members * P * sizeof(float), d->stream));
  COMPAR_CUDA_TRY(h2d(dx, X, static_cast<size_t>(rows) * kNumFeatures * sizeof(float)));
  COMPAR_CUDA_TRY(h2d(dt, T, static_cast<size_t>(rows) * kOutputs * sizeof(float)));
  COMPAR_CUDA_TRY(h2d(dmask, mask, static_cast<size_t>(rows) * kOutputs * sizeof(float)));
  COMPAR_CUDA_TRY(h2d(di, batch_idx, static_cast<size_t>(members) * steps * batch * sizeof(int)));
  rc = mlp_train_device(dp, dm, dv, members, dx, dt, dmask, di, steps, batch, lr, step0,
                        grads ? 0 : 1, dg, dl, d->stream);
  if (rc != COMPAR_OK) return rc;
  auto d2h = [&](void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, d->stream);
  };
  if (grads) {
    COMPAR_CUDA_TRY(d2h(grads, dg, members * P * sizeof(float)));
  } else {
    COMPAR_CUDA_TRY(d2h(params, dp, members * P * sizeof(float)));
    COMPAR_CUDA_TRY(d2h(adam_m, dm, members * P * sizeof(float)));
    COMPAR_CUDA_TRY(d2h(adam_v, dv, members * P * sizeof(float)));
  }
  if (loss) COMPAR_CUDA_TRY(d2h(loss, dl, static_cast<size_t>(members) * steps * sizeof(float)));
  COMPAR_CUDA_TRY(cudaStreamSynchronize(d->stream));
  return COMPAR_OK;
}

// Training from the records.  warm = continue from the current parameters
// and standardisation (fine-tuning); otherwise fresh statistics and a fresh
// initialisation.
static int train_impl(compar_ctx_t ctx, int steps, int batch, float lr, uint64_t seed, bool warm,
                      float* val_loss) {
  if (!ctx || steps <= 0 || batch <= 0 || batch > 128 || !(lr > 0)) return COMPAR_ERR_INVALID;
  if (ctx->host_only) return COMPAR_ERR_UNSUPPORTED;
  warm = warm && ctx->mlp.trained;
  // ---- assemble rows from the records (a fine-tune also rehearses the
  // sample of the records the loaded model was trained on)
  auto recs = ctx->rec.snapshot();
  if (warm) recs.insert(recs.end(), ctx->rehearsal.begin(), ctx->rehearsal.end());
  std::vector<std::array<float, kNumFeatures>> feats;
  std::vector<std::array<float, kOutputs>> tgt, msk;
  uint64_t st = seed ^ 0x5EEDull;
  // The records' own tolerance is not a property of the timing or the
  // error; each row gets a tolerance class drawn from the ones callers use,
  // so that the tolerance feature's training box spans them.
  const double tols[4] = {1e-6, 1e-5, 1e-3, 1e-1};
  for (const auto& r : recs) {
    if (r.variant < 0 || r.variant >= kNumVariants) continue;
    const bool has_t = r.time_ms > 0, has_e = r.rel_err > 0;
    if (!has_t && !has_e) continue;
    const double tol = tols[splitmix(st) % 4];
    feats.push_back(make_features(r.m, r.n, r.k, r.dtype, tol, std::max(1, r.batch)));
    std::array<float, kOutputs> t{}, m{};
    if (has_t) {
      // time head: log2 of measured / roofline-prior time (a learned correction)
      t[r.variant] = static_cast<float>(
          std::log2(static_cast<double>(r.time_ms)) -
          std::log2(prior_time_ms(r.variant, r.m, r.n, r.k, r.dtype, ctx->num_sms)));
      m[r.variant] = 1.f;
    }
    if (has_e) {
      t[kNumVariants + r.variant] =
          static_cast<float>(std::log10(std::max(1e-12, static_cast<double>(r.rel_err))));
      m[kNumVariants + r.variant] = 1.f;
    }
    tgt.push_back(t);
    msk.push_back(m);
  }
  const int rows = static_cast<int>(feats.size());
  if (rows < 16) return COMPAR_ERR_INVALID;
  // ---- standardisation statistics and training box
  MlpModel mm = ctx->mlp;
  for (int j = 0; j < kNumFeatures; ++j) {
    double s = 0, s2 = 0;
    float lo = INFINITY, hi = -INFINITY;
    for (const auto& f : feats) {
      s += f[j];
      s2 += static_cast<double>(f[j]) * f[j];
      lo = std::min(lo, f[j]);
      hi = std::max(hi, f[j]);
    }
    const double mean = s / rows;
    const double var = std::max(0.0, s2 / rows - mean * mean);
    if (warm) {  // the parameters were fitted to the current standardisation
      mm.feat_min[j] = std::min(mm.feat_min[j], lo);
      mm.feat_max[j] = std::max(mm.feat_max[j], hi);
      continue;
    }
    mm.feat_mean[j] = static_cast<float>(mean);
    mm.feat_std[j] = static_cast<float>(std::max(std::sqrt(var), 1e-3));
    mm.feat_min[j] = lo;
    mm.feat_max[j] = hi;
  }
  for (int o = 0; !warm && o < kOutputs; ++o) {
    double s = 0, s2 = 0, c = 0;
    for (int r = 0; r < rows; ++r)
      if (msk[r][o] > 0) {
        s += tgt[r][o];
        s2 += static_cast<double>(tgt[r][o]) * tgt[r][o];
        c += 1;
      }
    const double mean = c > 0 ? s / c : 0.0;
    const double var = c > 0 ? std::max(0.0, s2 / c - mean * mean) : 1.0;
    mm.out_mean[o] = static_cast<float>(mean);
    mm.out_std[o] = static_cast<float>(std::max(std::sqrt(var), 1e-2));
  }
  // ---- standardised arrays; 1 row in 10 held out for validation
  std::vector<float> X(static_cast<size_t>(rows) * kNumFeatures), T(static_cast<size_t>(rows) * kOutputs),
      M(static_cast<size_t>(rows) * kOutputs);
  std::vector<int> train_rows, val_rows;
  for (int r = 0; r < rows; ++r) {
    for (int j = 0; j < kNumFeatures; ++j)
      X[r * kNumFeatures + j] = (feats[r][j] - mm.feat_mean[j]) / mm.feat_std[j];
    for (int o = 0; o < kOutputs; ++o) {
      T[r * kOutputs + o] = msk[r][o] > 0 ? (tgt[r][o] - mm.out_mean[o]) / mm.out_std[o] : 0.f;
      M[r * kOutputs + o] = msk[r][o];
    }
    ((splitmix(st) % 10) == 0 ? val_rows : train_rows).push_back(r);
  }
  if (train_rows.empty()) return COMPAR_ERR_INVALID;
  // ---- initial parameters and bootstrap mini-batches per member
  const size_t P = MlpParams::count();
  std::vector<float> params(kEnsemble * P), flat;
  for (int e = 0; e < kEnsemble; ++e) {
    if (warm) {
      mm.members[e].flatten(flat);
    } else {
      MlpParams p;
      p.init(seed * 7919ull + 17ull * e + 1);
      p.flatten(flat);
    }
    std::copy(flat.begin(), flat.end(), params.begin() + e * P);
  }
  const int B = std::min<int>(batch, static_cast<int>(train_rows.size()));
  std::vector<int32_t> idx(static_cast<size_t>(kEnsemble) * steps * B);
  for (auto& i : idx) i = train_rows[splitmix(st) % train_rows.size()];
  std::vector<float> adam_m(kEnsemble * P, 0.f), adam_v(kEnsemble * P, 0.f);
  std::vector<float> losses(static_cast<size_t>(kEnsemble) * steps);
  // ---- validation loss (standardised masked MSE, mean over members) of a
  // parameter set on the held-out rows
  std::vector<float> vx(val_rows.size() * kNumFeatures);
  for (size_t i = 0; i < val_rows.size(); ++i)
    std::copy(X.begin() + val_rows[i] * kNumFeatures, X.begin() + (val_rows[i] + 1) * kNumFeatures,
              vx.begin() + i * kNumFeatures);
  auto val_loss_of = [&](const std::vector<float>& prm, double* out) -> int {
    std::vector<float> vy(val_rows.size() * kEnsemble * kOutputs);
    const int r = compar_mlp_forward(ctx, prm.data(), kEnsemble, vx.data(),
                                     static_cast<int>(val_rows.size()), vy.data());
    if (r != COMPAR_OK) return r;
    double num = 0, den = 0;
    for (int e = 0; e < kEnsemble; ++e)
      for (size_t i = 0; i < val_rows.size(); ++i)
        for (int o = 0; o < kOutputs; ++o) {
          const float mk = M[val_rows[i] * kOutputs + o];
          const float d = vy[(e * val_rows.size() + i) * kOutputs + o] - T[val_rows[i] * kOutputs + o];
          num += mk * d * d;
          den += mk;
        }
    *out = den > 0 ? num / den : 0.0;
    return COMPAR_OK;
  };
  // A fine-tune starts from weights that already fit most of these rows; it
  // is kept only if it lowers the held-out loss (live records and rehearsed
  // ones alike), so a fine-tune that drifts on a few new records is dropped.
  double vl_before = INFINITY;
  if (warm && !val_rows.empty()) {
    const int r = val_loss_of(params, &vl_before);
    if (r != COMPAR_OK) return r;
  }
  int rc = compar_mlp_train_steps(ctx, params.data(), adam_m.data(), adam_v.data(), kEnsemble,
                                  X.data(), T.data(), M.data(), rows, idx.data(), steps, B, lr,
                                  1, nullptr, losses.data());
  if (rc != COMPAR_OK) return rc;
  double vl = 0;
  if (!val_rows.empty()) {
    rc = val_loss_of(params, &vl);
    if (rc != COMPAR_OK) return rc;
  } else {
    vl = losses.back();
  }
  if (warm && !(vl < vl_before)) {
    if (val_loss) *val_loss = static_cast<float>(vl_before);
    return COMPAR_FINETUNE_KEPT;
  }
  for (int e = 0; e < kEnsemble; ++e) mm.members[e].unflatten(params.data() + e * P);
  if (val_loss) *val_loss = static_cast<float>(vl);
  mm.trained = true;
  ctx->mlp = mm;
  auto* d = static_cast<MlpDevice*>(ctx->mlp_dev);
  if (d) d->uploaded = false;
  ctx->decisions.clear();
  return COMPAR_OK;
}

int compar_selector_train(compar_ctx_t ctx, int steps, int batch, float lr, uint64_t seed,
                          float* val_loss) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  return train_impl(ctx, steps, batch, lr, seed, false, val_loss);
}

int compar_selector_finetune(compar_ctx_t ctx, int steps, int batch, float lr, uint64_t seed,
                             float* val_loss) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  const int rc = train_impl(ctx, steps, batch, lr, seed, true, val_loss);
  if (ctx && (rc == COMPAR_OK || rc == COMPAR_FINETUNE_KEPT)) ctx->online.retrains += 1;
  if (rc == COMPAR_FINETUNE_KEPT) {
    ctx->online.rejected += 1;
    return COMPAR_OK;
  }
  return rc;
}

int compar_set_online(compar_ctx_t ctx, double epsilon, int64_t retrain_every,
                      int finetune_steps) {
  if (!ctx || !(epsilon >= 0.0 && epsilon <= 1.0) || retrain_every < 0 || finetune_steps < 0)
    return COMPAR_ERR_INVALID;
  ctx->online.epsilon = epsilon;
  ctx->online.retrain_every = retrain_every;
  ctx->online.finetune_steps = finetune_steps;
  ctx->online.records_at_train =
      static_cast<int64_t>(ctx->rec.ring.size() + ctx->pending.size());
  if (epsilon > 0 || retrain_every > 0) ctx->rec.on = true;
  return COMPAR_OK;
}

int compar_online_stats(compar_ctx_t ctx, int64_t* explored, int64_t* retrains,
                        int64_t* rejected) {
  if (!ctx || !explored || !retrains) return COMPAR_ERR_INVALID;
  *explored = ctx->online.explored;
  *retrains = ctx->online.retrains;
  if (rejected) *rejected = ctx->online.rejected;
  return COMPAR_OK;
}

int compar_predict(compar_ctx_t ctx, int64_t m, int64_t n, int64_t k, compar_dtype_t dtype,
                   double tol, int batch, float* time_ms, float* rel_err, float* spread) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  if (!ctx || !time_ms || !rel_err || m <= 0 || n <= 0 || k <= 0 || batch < 1)
    return COMPAR_ERR_INVALID;
  if (!ctx->mlp.trained) return COMPAR_ERR_UNSUPPORTED;
  auto x = make_features(m, n, k, dtype, tol > 0 ? tol : 1e-5, batch);
  float out[kEnsemble * kOutputs];
  int rc = mlp_predict(ctx, x.data(), 1, out);
  if (rc != COMPAR_OK) return rc;
  for (int v = 0; v < kNumVariants; ++v) {
    double mt = 0, me = 0, s2 = 0;
    for (int e = 0; e < kEnsemble; ++e) {
      mt += out[e * kOutputs + v];
      me += out[e * kOutputs + kNumVariants + v];
    }
    mt /= kEnsemble;
    me /= kEnsemble;
    for (int e = 0; e < kEnsemble; ++e) {
      const double dd = out[e * kOutputs + v] - mt;
      s2 += dd * dd;
    }
    time_ms[v] = static_cast<float>(std::exp2(mt) * prior_time_ms(v, m, n, k, dtype, ctx->num_sms));
    rel_err[v] = static_cast<float>(std::pow(10.0, me));
    if (spread) spread[v] = static_cast<float>(std::sqrt(s2 / kEnsemble));
  }
  return COMPAR_OK;
}

}  // extern "C"
