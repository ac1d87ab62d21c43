// Cost and error models behind the variant choice: features, the error
// model, the history table, the roofline prior, the recorder and the MLP
// parameter container.  The paper's runtime chooses among variants with
// performance models learned from earlier runs and notes that more training
// of those models should improve the choice (Sec. 3.2, Sec. 5); the history
// table is that kind of model, the MLP (selector_mlp.cpp) the learned one.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <tuple>

#include "runtime.h"

namespace compar {

std::array<float, kNumFeatures> make_features(int64_t m, int64_t n, int64_t k, int dtype,
                                              double tol, int batch) {
  std::array<float, kNumFeatures> x{};
  x[0] = static_cast<float>(std::log2(static_cast<double>(std::max<int64_t>(m, 1))));
  x[1] = static_cast<float>(std::log2(static_cast<double>(std::max<int64_t>(n, 1))));
  x[2] = static_cast<float>(std::log2(static_cast<double>(std::max<int64_t>(k, 1))));
  x[3] = dtype == COMPAR_F32 ? 1.f : 0.f;
  x[4] = dtype == COMPAR_BF16 ? 1.f : 0.f;
  x[5] = dtype == COMPAR_F8E4M3 ? 1.f : 0.f;
  x[6] = static_cast<float>(std::log10(std::max(tol, 1e-12)));
  x[7] = static_cast<float>(std::log2(static_cast<double>(std::max(batch, 1))));
  return x;
}

// ------------------------------------------------------------- error model
// Defaults from the arithmetic of each variant (relative Frobenius error of
// a product of random inputs; u = 2^-24 is float32's unit roundoff):
//  * FP32 FMA variants and exact-product tensor-core variants on their own
//    input type: only accumulation error, ~ sqrt(k) u.
//  * TF32 on float32 inputs: operands keep 10 fraction bits, ~ 2^-11.
//  * BF16 on float32 inputs: operands rounded to 8 significant bits, ~ 2^-9.
//  * FP8 E4M3 on float32 inputs: 4 significant bits plus scaling, ~ 2^-5.
//  * 3xBF16 on float32 inputs: the split keeps ~16 bits and drops lo*lo.
//  * Tensor-core accumulation without promotion: the accumulator's additions
//    drop low bits (they do not round to nearest), so that part of the error
//    grows linearly in k: the c2 * k * u term.
ErrorModel::ErrorModel() {
  const float inf = INFINITY;
  for (auto& r : c0) r.fill(inf);
  for (auto& r : c1) r.fill(0.f);
  for (auto& r : c2) r.fill(0.f);
  // Constants fitted (with headroom) to errors measured on B300 against the
  // FP64 oracle for uniform[-1,1] and normal(0,1) inputs, k = 64 .. 16384:
  // naive FMA chain ~0.3 sqrt(k) u; SIMT below that; unpromoted tensor-core
  // accumulation ~0.018 k u; TF32 / BF16 / FP8 operand rounding of float32
  // inputs ~7-8e-4 / 2.4e-3 / 3.8e-2; promoted 3xBF16 flat at ~4.6e-6;
  // the 6-product split below SIMT's level.
  for (int v : {COMPAR_V_TC_TF32, COMPAR_V_TC_BF16, COMPAR_V_TC_FP8}) c2[v].fill(0.025f);
  for (int d = 0; d < 3; ++d) {
    c0[COMPAR_V_NAIVE][d] = 0.f;  c1[COMPAR_V_NAIVE][d] = 0.4f;
    c0[COMPAR_V_SIMT][d] = 0.f;   c1[COMPAR_V_SIMT][d] = 0.4f;
  }
  c0[COMPAR_V_TC_TF32][COMPAR_F32] = 7.8e-4f;
  c0[COMPAR_V_TC_BF16][COMPAR_F32] = 2.6e-3f;
  c0[COMPAR_V_TC_BF16][COMPAR_BF16] = 0.f;
  c0[COMPAR_V_TC_FP8][COMPAR_F32] = 4.2e-2f;
  c0[COMPAR_V_TC_FP8][COMPAR_F8E4M3] = 0.f;
  c0[COMPAR_V_SPLIT3][COMPAR_F32] = 5e-6f;
  c1[COMPAR_V_SPLIT3][COMPAR_F32] = 0.05f;
  // the fused variant computes the same products in the same order
  c0[COMPAR_V_SPLIT3_FUSED][COMPAR_F32] = 5e-6f;
  c1[COMPAR_V_SPLIT3_FUSED][COMPAR_F32] = 0.05f;
  // 6-product split: the pieces hold all 24 bits, the dropped terms are
  // ~2^-26 relative; what remains is FP32 accumulation of the promoted
  // per-stage partials (SIMT-like) and the tensor core's truncating adds.
  // Measured 6.2e-8 (k = 64) .. 4.1e-7 (k = 16384), ill-scaled columns alike.
  c0[COMPAR_V_SPLIT6][COMPAR_F32] = 6e-8f;
  c1[COMPAR_V_SPLIT6][COMPAR_F32] = 0.07f;
  // 3xTF32: 22-bit pieces and the dropped lo*lo term, ~2^-22 relative.
  // Measured 1.0e-7 (k = 64) .. 1.8e-7 (k = 16384), ill-scaled columns alike.
  c0[COMPAR_V_SPLIT3_TF32][COMPAR_F32] = 1.1e-7f;
  c1[COMPAR_V_SPLIT3_TF32][COMPAR_F32] = 0.07f;
}

double ErrorModel::predict(int v, int dtype, int64_t k) const {
  if (v < 0 || v >= kNumVariants || dtype < 0 || dtype > 2) return INFINITY;
  const double u = std::ldexp(1.0, -24);
  const double kk = static_cast<double>(std::max<int64_t>(k, 1));
  return c0[v][dtype] + c1[v][dtype] * std::sqrt(kk) * u + c2[v][dtype] * kk * u;
}

// ------------------------------------------------------------- history
bool HistKey::operator<(const HistKey& o) const {
  return std::tie(v, dtype, lm, ln, lk, batch) < std::tie(o.v, o.dtype, o.lm, o.ln, o.lk, o.batch);
}
bool HistKey::operator==(const HistKey& o) const {
  return v == o.v && dtype == o.dtype && lm == o.lm && ln == o.ln && lk == o.lk && batch == o.batch;
}

static int16_t qlog(int64_t x) {
  return static_cast<int16_t>(std::lround(4.0 * std::log2(static_cast<double>(std::max<int64_t>(x, 1)))));
}

HistKey HistoryModel::key(int v, int dtype, int64_t m, int64_t n, int64_t k, int batch) {
  HistKey h;
  h.v = static_cast<int8_t>(v);
  h.dtype = static_cast<int8_t>(dtype);
  h.lm = qlog(m);
  h.ln = qlog(n);
  h.lk = qlog(k);
  h.batch = static_cast<int8_t>(std::min(31, static_cast<int>(std::log2(std::max(batch, 1)))));
  return h;
}

void HistoryModel::observe(int v, int dtype, int64_t m, int64_t n, int64_t k, int batch, double ms) {
  HistVal& e = table[key(v, dtype, m, n, k, batch)];
  e.count += 1;
  const double d = ms - e.mean_ms;
  e.mean_ms += d / static_cast<double>(e.count);
  e.m2 += d * (ms - e.mean_ms);
  e.min_ms = std::min(e.min_ms, ms);
}

double HistoryModel::measured_min(int v, int dtype, int64_t m, int64_t n, int64_t k,
                                  int batch) const {
  auto it = table.find(key(v, dtype, m, n, k, batch));
  if (it == table.end() || it->second.count < 1 || !(it->second.min_ms > 0) ||
      !std::isfinite(it->second.min_ms))
    return -1;
  return it->second.min_ms;
}

double HistoryModel::predict(int v, int dtype, int64_t m, int64_t n, int64_t k, int batch,
                             bool* exact) const {
  const HistKey q = key(v, dtype, m, n, k, batch);
  if (exact) *exact = false;
  auto it = table.find(q);
  if (it != table.end()) {
    if (exact) *exact = true;
    return it->second.mean_ms;
  }
  // nearest neighbour among keys of the same variant / dtype / batch bucket
  HistKey lo = q, hi = q;
  lo.lm = lo.ln = lo.lk = INT16_MIN;
  hi.lm = hi.ln = hi.lk = INT16_MAX;
  int best = INT32_MAX;
  double best_ms = -1;
  for (auto i = table.lower_bound(lo); i != table.end() && !(hi < i->first); ++i) {
    const HistKey& h = i->first;
    if (h.batch != q.batch) continue;
    const int d = std::abs(h.lm - q.lm) + std::abs(h.ln - q.ln) + std::abs(h.lk - q.lk);
    if (d < best) {
      best = d;
      // scale by the work ratio 2^((dq)/4) per axis
      const double ratio = std::exp2((q.lm - h.lm + q.ln - h.ln + q.lk - h.lk) / 4.0);
      best_ms = i->second.mean_ms * ratio;
    }
  }
  if (best <= kMaxDist) return best_ms;
  return -1;
}

// ------------------------------------------------------------- roofline prior
double prior_time_ms(int v, int64_t m, int64_t n, int64_t k, int dtype, int num_sms) {
  const double M = static_cast<double>(m), N = static_cast<double>(n), K = static_cast<double>(k);
  const double bw = 6.0e12;  // bytes/s
  const double in_elem = dtype == COMPAR_F32 ? 4 : (dtype == COMPAR_BF16 ? 2 : 1);
  double flops = 2 * M * N * K, peak = 1, bytes = (M * K + K * N) * in_elem + M * N * 4;
  double ovh_us = 4;
  auto tiles = [&](int bm, int bn) {
    const double t = std::ceil(M / bm) * std::ceil(N / bn);
    return std::ceil(t / num_sms) * num_sms;  // wave quantisation
  };
  // The tensor-core variants' launch plan (compar_tc_plan): tiles of
  // 128 x 256 times the splits of K, in full waves of the SMs, each unit
  // running its own share of K; a split of K adds its in-cluster sum (up to
  // 8 splits) or its reduce launch.
  auto tc_units = [&](double* k_eff) {
    int64_t pl[9];
    if (tc_plan_info(v, m, n, k, num_sms, pl, false) != COMPAR_OK) {
      *k_eff = K;
      return tiles(128, 256);
    }
    const double splits = static_cast<double>(pl[2]);
    *k_eff = std::ceil(K / splits);
    if (splits > 1) ovh_us += splits <= 8 ? 1 : 4;
    return std::ceil(static_cast<double>(pl[1]) * splits / num_sms) * num_sms;
  };
  switch (v) {
    case COMPAR_V_NAIVE:
      peak = 4e12;
      // each output is one serial K-long FMA chain: with few outputs the
      // kernel is bound by that chain's latency (~60 ns per step measured)
      ovh_us += K * 0.06;
      break;
    case COMPAR_V_SIMT: {
      GemmCall g;  // contiguous operands at aligned addresses
      g.m = m;
      g.n = n;
      g.k = k;
      g.lda = k;
      g.ldb = n;
      g.ldc = n;
      g.dtype = static_cast<compar_dtype_t>(dtype);
      const SimtPlan pl = simt_plan(g, num_sms);
      if (pl.skinny) {
        // the skinny-M plan: B streamed once (~4.5 TB/s measured on long
        // chunks) overlapping FMAs on the rows padded to 8 or 16 (~30 TF/s)
        const double mp = m <= 8 ? 8.0 : std::ceil(M / 16) * 16;
        return 1e-3 * (8 + 1e6 * std::max(K * N * in_elem / 4.5e12, 2 * mp * N * K / 30e12));
      }
      // the tiled plan: bm x bn tiles times the splits of K in full waves,
      // each unit k_per long (32-row tiles run at a lower FMA rate)
      peak = pl.bm == 32 ? 35e12 : 45e12;
      const double units = std::ceil(M / pl.bm) * std::ceil(N / pl.bn) * pl.splits;
      flops = 2.0 * std::ceil(units / num_sms) * num_sms * pl.bm * pl.bn *
              static_cast<double>(pl.k_per);
      if (pl.splits > 1) ovh_us += 4;  // the reduce launch
      break;
    }
    case COMPAR_V_TC_TF32: {
      double ke;
      const double u = tc_units(&ke);
      peak = 0.8e15;
      flops = 2.0 * u * 128 * 256 * ke;
      bytes += K * N * 8;
      ovh_us += 8;
      break;
    }
    case COMPAR_V_TC_BF16: {
      double ke;
      const double u = tc_units(&ke);
      peak = 1.5e15;
      flops = 2.0 * u * 128 * 256 * ke;
      bytes += (dtype == COMPAR_F32 ? (M * K + K * N) * 6 : K * N * 4);
      ovh_us += 10;
      break;
    }
    case COMPAR_V_TC_FP8: {
      double ke;
      const double u = tc_units(&ke);
      peak = 3.0e15;
      flops = 2.0 * u * 128 * 256 * ke;
      bytes += (dtype == COMPAR_F32 ? (M * K + K * N) * 9 : K * N * 2);
      ovh_us += dtype == COMPAR_F32 ? 20 : 10;
      break;
    }
    case COMPAR_V_SPLIT3: {
      double ke;
      const double u = tc_units(&ke);
      peak = 1.5e15 / 3;
      flops = 2.0 * u * 128 * 256 * ke;
      bytes += (M * K + K * N) * 8;
      ovh_us += 10;
      break;
    }
    case COMPAR_V_SPLIT3_FUSED: {
      // no pre-pass: float32 operands read by the GEMM kernel itself
      double ke;
      const double u = tc_units(&ke);
      peak = 1.5e15 / 3;
      flops = 2.0 * u * 128 * 256 * ke;
      bytes += (M * K + K * N) * 4;
      ovh_us += 4;
      break;
    }
    case COMPAR_V_SPLIT6: {
      double ke;
      const double u = tc_units(&ke);
      peak = 1.5e15 / 6;
      flops = 2.0 * u * 128 * 256 * ke;
      bytes += (M * K + K * N) * 10;
      ovh_us += 12;
      break;
    }
    case COMPAR_V_SPLIT3_TF32: {
      double ke;
      const double u = tc_units(&ke);
      peak = 1.5e15 / 2 / 3;  // three products at the TF32 rate
      flops = 2.0 * u * 128 * 256 * ke;
      bytes += (M * K + K * N) * 12;
      ovh_us += 12;
      break;
    }
    default:
      return INFINITY;
  }
  return 1e3 * std::max(flops / peak, bytes / bw) + ovh_us * 1e-3;
}

// ------------------------------------------------------------- recorder
void Recorder::push(const compar_record_t& r) {
  if (static_cast<int64_t>(ring.size()) < kCap) {
    ring.push_back(r);
    size = static_cast<int64_t>(ring.size());
    head = 0;
    return;
  }
  ring[head] = r;  // full: overwrite the oldest
  head = (head + 1) % kCap;
}

std::vector<compar_record_t> Recorder::snapshot() const {
  std::vector<compar_record_t> out;
  out.reserve(ring.size());
  for (int64_t i = 0; i < static_cast<int64_t>(ring.size()); ++i)
    out.push_back(ring[(head + i) % ring.size()]);
  return out;
}

size_t DecisionKeyHash::operator()(const DecisionKey& d) const {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint64_t x) {
    h ^= x;
    h *= 1099511628211ull;
  };
  mix(static_cast<uint64_t>(d.m));
  mix(static_cast<uint64_t>(d.n));
  mix(static_cast<uint64_t>(d.k));
  mix(static_cast<uint64_t>(d.dtype));
  mix(static_cast<uint64_t>(d.tol_class));
  mix(static_cast<uint64_t>(d.batch));
  return static_cast<size_t>(h);
}

// ------------------------------------------------------------- MLP params
size_t MlpParams::count() {
  return static_cast<size_t>(kHidden) * kNumFeatures + kHidden + kHidden * kHidden + kHidden +
         static_cast<size_t>(kOutputs) * kHidden + kOutputs;
}

// He-uniform weights from a splitmix64 stream, zero biases.
void MlpParams::init(uint64_t seed) {
  uint64_t s = seed;
  auto next = [&]() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return static_cast<double>(z >> 11) * (1.0 / 9007199254740992.0);  // [0,1)
  };
  auto fill = [&](std::vector<float>& w, int o, int i) {
    w.resize(static_cast<size_t>(o) * i);
    const double bound = std::sqrt(6.0 / i);
    for (auto& x : w) x = static_cast<float>((2 * next() - 1) * bound);
  };
  fill(W1, kHidden, kNumFeatures);
  b1.assign(kHidden, 0.f);
  fill(W2, kHidden, kHidden);
  b2.assign(kHidden, 0.f);
  fill(W3, kOutputs, kHidden);
  b3.assign(kOutputs, 0.f);
}

void MlpParams::flatten(std::vector<float>& out) const {
  out.clear();
  out.reserve(count());
  for (auto* v : {&W1, &b1, &W2, &b2, &W3, &b3}) out.insert(out.end(), v->begin(), v->end());
}

void MlpParams::unflatten(const float* p) {
  auto take = [&](std::vector<float>& v, size_t n) {
    v.assign(p, p + n);
    p += n;
  };
  take(W1, static_cast<size_t>(kHidden) * kNumFeatures);
  take(b1, kHidden);
  take(W2, static_cast<size_t>(kHidden) * kHidden);
  take(b2, kHidden);
  take(W3, static_cast<size_t>(kOutputs) * kHidden);
  take(b3, kOutputs);
}

}  // namespace compar
