// GEMM on host matrices (compar_gemm_host): the library moves A, B (and C
// when beta != 0) to the device, runs the selected variant and brings C back,
// overlapping the transfers with the products.
//
// Per call: B goes up first (every panel needs all of it); A and C then move
// in row panels on two internal copy streams, and each panel is one
// selected-variant GEMM on the caller's stream, so the upload of panel p+1
// and the download of panel p-1 overlap the product of panel p.  Device
// buffers come in two sets used by alternate calls: the uploads of a call
// wait only for the call before the previous one, so they overlap the
// previous call's products as well.  (Hence the host inputs are read from
// the moment of the call, not from the point the stream has reached.)  The
// caller's stream waits for every download, so when it reaches the end of
// the call C is in host memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "runtime.h"

namespace compar {

int gemm_call(compar_ctx* ctx, GemmCall& c, cudaStream_t s);

namespace {

constexpr int kSlots = 2;
constexpr int kMaxPanels = 8;
constexpr int64_t kMinPanelRows = 1024;

struct Slot {
  void* dA = nullptr;
  void* dB = nullptr;
  float* dC = nullptr;
  size_t a_bytes = 0, b_bytes = 0, c_bytes = 0;
  cudaEvent_t done = nullptr;  // recorded on the caller's stream at the end of its last call
  bool used = false;
};

struct HostIO {
  Slot slot[kSlots];
  int next = 0;
  cudaStream_t up = nullptr, down = nullptr;
  cudaEvent_t ev_up[kMaxPanels] = {}, ev_mm[kMaxPanels] = {}, ev_dn[kMaxPanels] = {};
};

HostIO* state(compar_ctx* ctx) { return static_cast<HostIO*>(ctx->hostio_state); }

int make_event(cudaEvent_t* e) {
  if (*e) return COMPAR_OK;
  COMPAR_CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  return COMPAR_OK;
}

int ensure_state(compar_ctx* ctx, HostIO** out) {
  HostIO* h = state(ctx);
  if (!h) {
    h = new HostIO();
    ctx->hostio_state = h;
  }
  if (!h->up) COMPAR_CUDA_TRY(cudaStreamCreateWithFlags(&h->up, cudaStreamNonBlocking));
  if (!h->down) COMPAR_CUDA_TRY(cudaStreamCreateWithFlags(&h->down, cudaStreamNonBlocking));
  int rc = COMPAR_OK;
  for (int i = 0; rc == COMPAR_OK && i < kMaxPanels; ++i) {
    rc = make_event(&h->ev_up[i]);
    if (rc == COMPAR_OK) rc = make_event(&h->ev_mm[i]);
    if (rc == COMPAR_OK) rc = make_event(&h->ev_dn[i]);
  }
  for (int i = 0; rc == COMPAR_OK && i < kSlots; ++i) rc = make_event(&h->slot[i].done);
  *out = h;
  return rc;
}

// Grows one device buffer of a slot.  The slot's previous call has finished
// on the device when this runs (the caller synchronised on its event).
int grow(void** p, size_t* have, size_t need) {
  if (*have >= need) return COMPAR_OK;
  if (*p) COMPAR_CUDA_TRY(cudaFree(*p));
  *p = nullptr;
  *have = 0;
  COMPAR_CUDA_TRY(cudaMalloc(p, need));
  *have = need;
  return COMPAR_OK;
}

size_t elem_size(compar_dtype_t d) { return d == COMPAR_F32 ? 4 : (d == COMPAR_BF16 ? 2 : 1); }

}  // namespace

void hostio_release(compar_ctx* ctx) {
  HostIO* h = state(ctx);
  if (!h) return;
  for (auto& sl : h->slot) {
    cudaFree(sl.dA);
    cudaFree(sl.dB);
    cudaFree(sl.dC);
    if (sl.done) cudaEventDestroy(sl.done);
  }
  for (int i = 0; i < kMaxPanels; ++i) {
    if (h->ev_up[i]) cudaEventDestroy(h->ev_up[i]);
    if (h->ev_mm[i]) cudaEventDestroy(h->ev_mm[i]);
    if (h->ev_dn[i]) cudaEventDestroy(h->ev_dn[i]);
  }
  if (h->up) cudaStreamDestroy(h->up);
  if (h->down) cudaStreamDestroy(h->down);
  delete h;
  ctx->hostio_state = nullptr;
}

int gemm_host(compar_ctx* ctx, GemmCall base, const void* hA, const void* hB, float* hC,
              cudaStream_t s) {
  HostIO* h = nullptr;
  int rc = ensure_state(ctx, &h);
  if (rc != COMPAR_OK) return rc;
  const int64_t m = base.m, n = base.n, k = base.k;
  const size_t es = elem_size(base.dtype);
  const bool read_c = base.beta != 0.f;
  Slot& sl = h->slot[h->next];
  h->next = (h->next + 1) % kSlots;

  const size_t need_a = static_cast<size_t>(m) * k * es, need_b = static_cast<size_t>(k) * n * es;
  const size_t need_c = static_cast<size_t>(m) * n * sizeof(float);
  if (sl.a_bytes < need_a || sl.b_bytes < need_b || sl.c_bytes < need_c) {
    // the slot's earlier call must be finished before its buffers go
    if (sl.used) COMPAR_CUDA_TRY(cudaEventSynchronize(sl.done));
    rc = grow(&sl.dA, &sl.a_bytes, need_a);
    if (rc == COMPAR_OK) rc = grow(&sl.dB, &sl.b_bytes, need_b);
    if (rc == COMPAR_OK) rc = grow(reinterpret_cast<void**>(&sl.dC), &sl.c_bytes, need_c);
    if (rc != COMPAR_OK) return rc;
  }

  // Uploads into this slot wait for the slot's previous call to finish.
  if (sl.used) {
    COMPAR_CUDA_TRY(cudaStreamWaitEvent(h->up, sl.done, 0));
    COMPAR_CUDA_TRY(cudaStreamWaitEvent(h->down, sl.done, 0));
  }
  if (need_b > 0)
    COMPAR_CUDA_TRY(cudaMemcpyAsync(sl.dB, hB, need_b, cudaMemcpyHostToDevice, h->up));

  // Row panels: at least kMinPanelRows rows each, at most kMaxPanels.
  const int panels =
      static_cast<int>(std::clamp<int64_t>(m / kMinPanelRows, 1, static_cast<int64_t>(kMaxPanels)));
  const int64_t rows_per = (m + panels - 1) / panels;
  for (int p = 0; p < panels; ++p) {
    const int64_t r0 = p * rows_per;
    const int64_t rows = std::min<int64_t>(rows_per, m - r0);
    if (rows <= 0) break;
    uint8_t* dA = static_cast<uint8_t*>(sl.dA) + static_cast<size_t>(r0) * k * es;
    float* dC = sl.dC + static_cast<size_t>(r0) * n;
    const uint8_t* srcA = static_cast<const uint8_t*>(hA) + static_cast<size_t>(r0) * k * es;
    float* hCp = hC + static_cast<size_t>(r0) * n;
    if (k > 0)
      COMPAR_CUDA_TRY(cudaMemcpyAsync(dA, srcA, static_cast<size_t>(rows) * k * es,
                                      cudaMemcpyHostToDevice, h->up));
    if (read_c)
      COMPAR_CUDA_TRY(cudaMemcpyAsync(dC, hCp, static_cast<size_t>(rows) * n * sizeof(float),
                                      cudaMemcpyHostToDevice, h->up));
    COMPAR_CUDA_TRY(cudaEventRecord(h->ev_up[p], h->up));
    COMPAR_CUDA_TRY(cudaStreamWaitEvent(s, h->ev_up[p], 0));
    GemmCall c = base;
    c.m = rows;
    c.lda = k;
    c.ldb = n;
    c.ldc = n;
    c.A = dA;
    c.B = sl.dB;
    c.C = dC;
    rc = gemm_call(ctx, c, s);
    if (rc != COMPAR_OK) {
      // leave the streams consistent: nothing later on `s` may overtake the
      // copies already queued for this slot
      cudaEventRecord(sl.done, h->up);
      cudaStreamWaitEvent(s, sl.done, 0);
      sl.used = true;
      return rc;
    }
    COMPAR_CUDA_TRY(cudaEventRecord(h->ev_mm[p], s));
    COMPAR_CUDA_TRY(cudaStreamWaitEvent(h->down, h->ev_mm[p], 0));
    COMPAR_CUDA_TRY(cudaMemcpyAsync(hCp, dC, static_cast<size_t>(rows) * n * sizeof(float),
                                    cudaMemcpyDeviceToHost, h->down));
    COMPAR_CUDA_TRY(cudaEventRecord(h->ev_dn[p], h->down));
  }
  // The call ends on `s` once every panel of C is in host memory.
  for (int p = 0; p < panels; ++p) {
    if (p * rows_per >= m) break;
    COMPAR_CUDA_TRY(cudaStreamWaitEvent(s, h->ev_dn[p], 0));
  }
  COMPAR_CUDA_TRY(cudaEventRecord(sl.done, s));
  sl.used = true;
  return COMPAR_OK;
}

}  // namespace compar
