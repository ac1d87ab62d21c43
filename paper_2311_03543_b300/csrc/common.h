// Internal declarations shared by the host-side parts of libcompar.
// Nothing here is part of the public C ABI (include/compar.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "compar.h"

namespace compar {

#define COMPAR_CUDA_TRY(expr)                                              \
  do {                                                                     \
    cudaError_t e__ = (expr);                                              \
    if (e__ != cudaSuccess) {                                              \
      compar::set_last_cuda_error(e__, #expr, __FILE__, __LINE__);         \
      return COMPAR_ERR_CUDA;                                              \
    }                                                                      \
  } while (0)

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// Per-call description used by eligibility, selection and launch.
struct GemmCall {
  int64_t m = 0, n = 0, k = 0;
  int64_t lda = 0, ldb = 0, ldc = 0;
  compar_dtype_t dtype = COMPAR_F32;
  double tol = 0;
  const void* A = nullptr;
  const void* B = nullptr;
  float* C = nullptr;
  float alpha = 1.f, beta = 0.f;
  float scale_a = 1.f, scale_b = 1.f;  // fp8 input dequantisation factors
  int batch = 1;
};

// Device scratch owned by a context, grown stream-ordered.
struct Workspace {
  void* ptr = nullptr;
  size_t bytes = 0;
  // Arrival counters: each word holds the epoch of the launch that last
  // counted on it (high 32 bits) and that launch's count (low 32 bits).  A
  // launch takes a fresh epoch (never 0), so a word from any earlier launch
  // reads as a count of zero: nothing has to be reset between calls, and a
  // word left inconsistent by calls that overlapped on the GPU does not
  // carry over into later calls.  Grown zeroed, stream-ordered.
  unsigned long long* counters = nullptr;
  size_t counter_n = 0;
  uint32_t counter_epoch = 0;
  uint32_t next_epoch() {
    if (++counter_epoch == 0) counter_epoch = 1;
    return counter_epoch;
  }
  int ensure(size_t need, cudaStream_t s);
  int ensure_counters(size_t n, cudaStream_t s);
  // Counter words [0, n) for one launch, with a fresh epoch in *epoch.  When
  // `s` is being captured into a graph, the words are also zeroed in the
  // captured work: every replay of the graph runs the same epoch, so each
  // must start from zero counts.
  int take_counters(size_t n, cudaStream_t s, uint32_t* epoch);
  void release();
};

// ------------------------------------------------------------- profiling
// Optional CUDA-event timing of the main GEMM kernel of each call (not its
// pre-passes), accumulated per variant and resolved lazily.
// Slots 0..COMPAR_V_COUNT-1: GEMM variant ids; kStencilProfileBase + s:
// stencil variant s.
constexpr int kStencilProfileBase = COMPAR_V_COUNT;
struct KernelProfiler {
  static constexpr int kSlots = 16;
  bool on = false;
  struct Pend {
    cudaEvent_t a, b;
    int v;
  };
  std::vector<cudaEvent_t> pool;
  std::vector<Pend> pend;
  static_assert(kStencilProfileBase + COMPAR_S_COUNT <= 16, "profiler slots");
  double total_ms[kSlots] = {};
  int64_t launches[kSlots] = {};
  cudaEvent_t begin(cudaStream_t s);
  void end(cudaEvent_t a, cudaStream_t s, int v);
  void resolve();
  void reset();
  void release();
};

// Process-wide count of kernels this library launched.
void count_launch(int n = 1);
int64_t launch_count();

// ------------------------------------------------------------- kernel entry
// Each returns a compar_status_t; all are asynchronous on `s`.
struct DeviceGuard {  // device error word + wait budget handed to kernels
  int* err_word = nullptr;
  unsigned long long budget_ns = 2000000000ull;
  KernelProfiler* prof = nullptr;
  // tensor-core variants on CTA pairs: -1 automatic, 0 never, 1 always
  int tc_pair = -1;
};

// One process may drive several GPUs (one context each), so one-time kernel
// set-up (shared-memory opt-ins, occupancy queries) is kept per device.
constexpr int kMaxDevices = 64;

// The calling thread's current device, or -1 when there is none or it is
// numbered kMaxDevices or above.
int current_device_index();

// Raises `func`'s dynamic shared-memory limit to `bytes` on the current
// device, once per (device, kernel, size).
cudaError_t smem_opt_in(const void* func, int bytes);

// Makes a context's device current for one API call and puts the caller's
// device back when the call returns.  Does nothing when that device is
// already current, or for device -1 (host-only contexts).  It also clears a
// non-sticky CUDA error the caller left pending, which the call's launch
// checks would otherwise read as their own.
// COMPAR_OK, or COMPAR_ERR_UNSUPPORTED (with the error text) when `s` is being
// captured into a CUDA graph: for calls that synchronise or run a graph of
// their own.
int refuse_capture(cudaStream_t s, const char* call);

class DeviceScope {
 public:
  explicit DeviceScope(int device);
  ~DeviceScope();
  DeviceScope(const DeviceScope&) = delete;
  DeviceScope& operator=(const DeviceScope&) = delete;

 private:
  int prev_ = -1;
  bool switched_ = false;
};

int launch_naive(const GemmCall& c, const DeviceGuard& g, cudaStream_t s);
int launch_simt(const GemmCall& c, Workspace& ws, const DeviceGuard& g, int num_sms,
                cudaStream_t s);
int launch_scale_c(float* C, int64_t m, int64_t n, int64_t ldc, float beta, cudaStream_t s);
// C = alpha * sum over s < splits of partial[s][m][n] + beta * C.
int launch_splitk_reduce(int m, int n, int splits, const float* partial, float alpha, float beta,
                         float* C, int64_t ldc, int num_sms, cudaStream_t s);
// Tile shape and split-K plan of the SIMT variant: each output is the sum
// of `splits` partial dot products, each at most `k_per` terms long.
// Launch plan of the SIMT variant: the tiled kernel (bm x bn tiles, K split
// `splits` ways), or the skinny kernel (row groups of bm = 8 or 16,
// 512-column blocks, K chunks of k_per summed in clusters of `cluster`,
// `splits` cluster sums added by the reduce pass).  k_per is the longest FMA
// chain.
struct SimtPlan {
  int bm = 0, bn = 0, bk = 0;
  int splits = 1;
  int64_t k_per = 0;
  bool skinny = false;
  int cluster = 1;
};
SimtPlan simt_plan(const GemmCall& c, int num_sms);
int launch_simt_scratch(const GemmCall& c, float* scratch, size_t scratch_bytes, int num_sms,
                        cudaStream_t s, size_t* need_bytes);
void set_last_error_text(const std::string& text);

// Tensor-core variants (tcgen05).  kind: COMPAR_V_TC_TF32 / TC_BF16 / TC_FP8 / SPLIT3 /
// SPLIT6.
int launch_tc(int variant, const GemmCall& c, Workspace& ws, const DeviceGuard& g,
              int num_sms, cudaStream_t s);
bool tc_supported(int variant, const GemmCall& c);
int tc_plan_info(int variant, int64_t m, int64_t n, int64_t k, int slots, int64_t* out,
                 bool pair);

int launch_timeout_selftest(const DeviceGuard& g, cudaStream_t s);
// One-thread kernel that holds `s` until *flag_dev (host-mapped) reaches
// `ticket` or 2 ms pass: put before a recorded call's launches so that they
// run back to back once the host has enqueued them all.
int launch_record_gate(const unsigned int* flag_dev, unsigned int ticket, cudaStream_t s);

// Pre-pass kernels (prepass.cu).
int prepass_convert(const void* X, compar_dtype_t in_t, int64_t rows, int64_t cols,
                    int64_t ldx, void* Y, int out_kind, int64_t ldy, bool transpose,
                    void* Y_lo, const float* dscale, int num_sms, cudaStream_t s);
// One float32 matrix of a row-wise convert: rows x cols of X (pitch ldx)
// into Y (and Y_lo for the splits; pitch ldy), scaled by *dscale (fp8).
struct RowConvert {
  const float* X;
  int64_t rows, cols, ldx;
  void* Y;
  void* Y_lo;
  int64_t ldy;
  const float* dscale;
};
// Row-wise converts of two float32 matrices (out_kind PP_BF16 or a split)
// in one launch of the vectorised row kernel, launched programmatically (it
// waits for the stream's previous kernel before touching memory).
// COMPAR_ERR_UNSUPPORTED, with nothing launched, when either matrix misses
// the kernel's rules (cols % 8 == 0, 16-byte rows and bases): the caller
// then converts them one by one with prepass_convert.
int prepass_convert_rows2(const RowConvert& a, const RowConvert& b, int out_kind, int num_sms,
                          cudaStream_t s);
// amax(|X|) and amax(|Y|) in one launch, as per-block maxima: block b
// writes d_block_max[2 b] and [2 b + 1]; at most max_blocks blocks, the
// number used in *nblocks (0 when both are empty).
int prepass_amax2(const float* X, int64_t xr, int64_t xc, int64_t ldx, const float* Y, int64_t yr,
                  int64_t yc, int64_t ldy, float* d_block_max, int max_blocks, int num_sms,
                  int* nblocks, cudaStream_t s);
// {s_x, 1/s_x, s_y, 1/s_y} with s = 448 / amax (1 when amax == 0), the
// amaxes reduced from prepass_amax2's per-block maxima.
int prepass_fp8_scales(const float* d_block_max, int nblocks, float* d_out, cudaStream_t s);

// out_kind values for prepass_convert.  The split kinds write piece p of
// element idx at Y + p * (Y_lo - Y) (pieces equally spaced, Y_lo = piece 1):
//   PP_SPLIT_BF16    hi = bf16(x), lo = bf16(x - hi)
//   PP_SPLIT_BF16_3P hi = bf16(x), mid = bf16(x - hi), lo = bf16(x - hi - mid)
//   PP_SPLIT_TF32    hi = tf32(x), lo = tf32(x - hi) (float32 pieces, RNA)
enum PrepassOut {
  PP_F32 = 0,
  PP_BF16 = 1,
  PP_SPLIT_BF16 = 2,
  PP_E4M3 = 3,
  PP_COPY = 4,
  PP_SPLIT_BF16_3P = 5,
  PP_SPLIT_TF32 = 6
};

// Thermal stencil (stencil.cu).  `tmp` is a rows x cols scratch grid;
// aligned16: T_in, P, T_out and tmp are 16-byte aligned.
int stencil_launch(int v, int64_t rows, int64_t cols, int iters,
                   const compar_stencil_params_t& prm, const float* T_in, const float* P,
                   float* T_out, float* tmp, const DeviceGuard& g, cudaStream_t s);
bool stencil_supported(int v, int64_t rows, int64_t cols, bool aligned16);

// TMA tensor-map encoding (tma.cpp).
bool tma_available();
int tma_encode_2d(CUtensorMap* map, CUtensorMapDataType dt, int elem_bytes, const void* base,
                  uint64_t inner, uint64_t outer, uint64_t ld_elems, uint32_t box_inner,
                  uint32_t box_outer, int swizzle_bytes = 128);

std::string last_error_text();

}  // namespace compar
