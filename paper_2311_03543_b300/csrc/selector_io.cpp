// Selector files: the persisted state of the cost models (history table,
// error model, MLP ensemble and feature normaliser, grouped tile choice,
// stencil history table).
// The paper's runtime keeps its performance models across runs; this is the
// equivalent checkpoint.  Format (little endian):
//   "CMPRSEL1" | u32 version | u64 payload bytes | payload | u64 FNV-1a(payload)
// The payload ends with a rehearsal sample of timing records (up to
// kRehearsal, drawn uniformly from the training records and any sample
// loaded before) for online fine-tuning.
// A file that fails any check leaves the loaded models untouched.
#include <cmath>
#include <cstring>
#include <fstream>
#include <vector>

#include "runtime.h"

namespace compar {
namespace {

constexpr char kMagic[8] = {'C', 'M', 'P', 'R', 'S', 'E', 'L', '1'};
constexpr uint32_t kVersion = 8;  // 8: fastest time per history entry; 7 (read too): rehearsal records; variant ids 0..9 (20 MLP outputs)
constexpr size_t kRehearsal = 16384;

uint64_t fnv1a(const uint8_t* p, size_t n) {
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

struct Writer {
  std::vector<uint8_t> b;
  template <typename T>
  void put(const T& v) {
    const auto* p = reinterpret_cast<const uint8_t*>(&v);
    b.insert(b.end(), p, p + sizeof(T));
  }
  void put_floats(const std::vector<float>& v) {
    const auto* p = reinterpret_cast<const uint8_t*>(v.data());
    b.insert(b.end(), p, p + v.size() * sizeof(float));
  }
};

struct Reader {
  const uint8_t* p;
  size_t n, off = 0;
  bool ok = true;
  template <typename T>
  T get() {
    T v{};
    if (off + sizeof(T) > n) {
      ok = false;
      return v;
    }
    memcpy(&v, p + off, sizeof(T));
    off += sizeof(T);
    return v;
  }
  void get_floats(float* dst, size_t count) {
    if (off + count * sizeof(float) > n) {
      ok = false;
      return;
    }
    memcpy(dst, p + off, count * sizeof(float));
    off += count * sizeof(float);
  }
};

// History tables: count, then (key, running mean, M2, count, fastest) per
// entry (version 7 files have no fastest time: it is read as the mean).
void put_hist(Writer& w, const HistoryModel& h) {
  w.put<uint32_t>(static_cast<uint32_t>(h.table.size()));
  for (const auto& kv : h.table) {
    w.put(kv.first.v);
    w.put(kv.first.dtype);
    w.put(kv.first.lm);
    w.put(kv.first.ln);
    w.put(kv.first.lk);
    w.put(kv.first.batch);
    w.put(kv.second.mean_ms);
    w.put(kv.second.m2);
    w.put(kv.second.count);
    w.put(kv.second.min_ms);
  }
}

void get_hist(Reader& r, HistoryModel& h, int num_variants, uint32_t version) {
  const uint32_t n = r.get<uint32_t>();
  for (uint32_t i = 0; r.ok && i < n; ++i) {
    HistKey k;
    k.v = r.get<int8_t>();
    k.dtype = r.get<int8_t>();
    k.lm = r.get<int16_t>();
    k.ln = r.get<int16_t>();
    k.lk = r.get<int16_t>();
    k.batch = r.get<int8_t>();
    HistVal v;
    v.mean_ms = r.get<double>();
    v.m2 = r.get<double>();
    v.count = r.get<int64_t>();
    v.min_ms = version >= 8 ? r.get<double>() : v.mean_ms;
    if (k.v < 0 || k.v >= num_variants || k.dtype < 0 || k.dtype > 2) r.ok = false;
    h.table[k] = v;
  }
}

}  // namespace
}  // namespace compar

using namespace compar;

extern "C" int compar_selector_save(compar_ctx_t ctx, const char* path) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  if (!ctx || !path) return COMPAR_ERR_INVALID;
  Writer w;
  put_hist(w, ctx->hist);
  for (const auto& r : ctx->err.c0) for (float x : r) w.put(x);
  for (const auto& r : ctx->err.c1) for (float x : r) w.put(x);
  for (const auto& r : ctx->err.c2) for (float x : r) w.put(x);
  w.put(ctx->err.margin);
  const MlpModel& mm = ctx->mlp;
  w.put<uint8_t>(mm.trained ? 1 : 0);
  for (float x : mm.feat_mean) w.put(x);
  for (float x : mm.feat_std) w.put(x);
  for (float x : mm.feat_min) w.put(x);
  for (float x : mm.feat_max) w.put(x);
  for (float x : mm.out_mean) w.put(x);
  for (float x : mm.out_std) w.put(x);
  w.put(mm.conf_std);
  w.put(mm.box_slack);
  w.put<uint32_t>(static_cast<uint32_t>(MlpParams::count()));
  std::vector<float> flat;
  for (const auto& m : mm.members) {
    if (mm.trained) {
      m.flatten(flat);
    } else {
      flat.assign(MlpParams::count(), 0.f);
    }
    w.put_floats(flat);
  }
  w.put<uint32_t>(static_cast<uint32_t>(ctx->batched_cfg.size()));
  for (const auto& kv : ctx->batched_cfg) {
    w.put<uint64_t>(kv.first);
    w.put<int32_t>(kv.second);
  }
  put_hist(w, ctx->stencil.hist);
  {
    // rehearsal sample: reservoir over the loaded sample and the live records
    std::vector<compar_record_t> pool = ctx->rehearsal;
    const auto live = ctx->rec.snapshot();
    pool.insert(pool.end(), live.begin(), live.end());
    uint64_t st = 0x9E3779B97F4A7C15ull ^ pool.size();
    auto next = [&]() {
      uint64_t z = (st += 0x9E3779B97F4A7C15ull);
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      return z ^ (z >> 31);
    };
    for (size_t i = pool.size(); i > 1 && pool.size() > kRehearsal; --i)
      std::swap(pool[i - 1], pool[next() % i]);  // shuffle, then keep the first kRehearsal
    if (pool.size() > kRehearsal) pool.resize(kRehearsal);
    w.put<uint32_t>(static_cast<uint32_t>(pool.size()));
    for (const auto& rec : pool) w.put(rec);
  }

  std::ofstream f(path, std::ios::binary | std::ios::trunc);
  if (!f) return COMPAR_ERR_IO;
  const uint64_t nbytes = w.b.size();
  const uint64_t sum = fnv1a(w.b.data(), w.b.size());
  f.write(kMagic, 8);
  f.write(reinterpret_cast<const char*>(&kVersion), 4);
  f.write(reinterpret_cast<const char*>(&nbytes), 8);
  f.write(reinterpret_cast<const char*>(w.b.data()), static_cast<std::streamsize>(w.b.size()));
  f.write(reinterpret_cast<const char*>(&sum), 8);
  return f.good() ? COMPAR_OK : COMPAR_ERR_IO;
}

extern "C" int compar_selector_load(compar_ctx_t ctx, const char* path) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  if (!ctx || !path) return COMPAR_ERR_INVALID;
  std::ifstream f(path, std::ios::binary);
  if (!f) return COMPAR_ERR_IO;
  std::vector<uint8_t> all((std::istreambuf_iterator<char>(f)), std::istreambuf_iterator<char>());
  if (all.size() < 8 + 4 + 8 + 8) return COMPAR_ERR_IO;
  if (memcmp(all.data(), kMagic, 8) != 0) return COMPAR_ERR_IO;
  uint32_t version;
  uint64_t nbytes, sum;
  memcpy(&version, all.data() + 8, 4);
  memcpy(&nbytes, all.data() + 12, 8);
  if (version != kVersion && version != 7) return COMPAR_ERR_IO;
  if (nbytes != all.size() - 28) return COMPAR_ERR_IO;
  const uint8_t* payload = all.data() + 20;
  memcpy(&sum, payload + nbytes, 8);
  if (fnv1a(payload, nbytes) != sum) return COMPAR_ERR_IO;

  Reader r{payload, nbytes};
  HistoryModel hist;
  get_hist(r, hist, kNumVariants, version);
  ErrorModel err;
  for (auto& row : err.c0) for (float& x : row) x = r.get<float>();
  for (auto& row : err.c1) for (float& x : row) x = r.get<float>();
  for (auto& row : err.c2) for (float& x : row) x = r.get<float>();
  err.margin = r.get<float>();
  if (!(err.margin >= 1.0f) || !std::isfinite(err.margin)) r.ok = false;
  MlpModel mm;
  mm.trained = r.get<uint8_t>() != 0;
  for (float& x : mm.feat_mean) x = r.get<float>();
  for (float& x : mm.feat_std) x = r.get<float>();
  for (float& x : mm.feat_min) x = r.get<float>();
  for (float& x : mm.feat_max) x = r.get<float>();
  for (float& x : mm.out_mean) x = r.get<float>();
  for (float& x : mm.out_std) x = r.get<float>();
  mm.conf_std = r.get<float>();
  mm.box_slack = r.get<float>();
  const uint32_t np = r.get<uint32_t>();
  if (np != MlpParams::count()) r.ok = false;
  std::vector<float> flat(MlpParams::count());
  for (auto& m : mm.members) {
    if (!r.ok) break;
    r.get_floats(flat.data(), flat.size());
    m.unflatten(flat.data());
  }
  std::unordered_map<uint64_t, int> batched;
  const uint32_t nb = r.get<uint32_t>();
  for (uint32_t i = 0; r.ok && i < nb; ++i) {
    const uint64_t sig = r.get<uint64_t>();
    const int32_t cfg = r.get<int32_t>();
    if (cfg < 0 || cfg > 4) r.ok = false;
    batched[sig] = cfg;
  }
  HistoryModel stencil_hist;
  get_hist(r, stencil_hist, COMPAR_S_COUNT, version);
  const uint32_t nr = r.get<uint32_t>();
  if (nr > kRehearsal) r.ok = false;
  std::vector<compar_record_t> rehearsal;
  for (uint32_t i = 0; r.ok && i < nr; ++i) {
    const auto rec = r.get<compar_record_t>();
    if (rec.variant < 0 || rec.variant >= kNumVariants || rec.m < 1 || rec.n < 1 || rec.k < 1)
      r.ok = false;
    rehearsal.push_back(rec);
  }
  if (!r.ok || r.off != nbytes) return COMPAR_ERR_IO;

  ctx->hist = std::move(hist);
  ctx->err = err;
  ctx->mlp = mm;
  ctx->batched_cfg = std::move(batched);
  ctx->stencil.hist = std::move(stencil_hist);
  ctx->rehearsal = std::move(rehearsal);
  ctx->stencil.decisions.clear();
  ctx->decisions.clear();
  mlp_release(ctx);  // device copies of the old weights are stale
  return COMPAR_OK;
}
