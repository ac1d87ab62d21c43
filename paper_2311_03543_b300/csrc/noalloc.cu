// compar_gemm_simt_noalloc: the FP32 SIMT GEMM variant for callers that
// cannot allocate device memory.
//
// Some callers may not call cudaMalloc (or anything that allocates) at the
// point where they need a GEMM: code that runs inside a host application or
// framework that owns every byte of device memory through its own pool, a
// latency-critical path that cannot afford the implicit synchronisation an
// allocation can cause, or a plug-in whose host never gave it an allocator.
// The regular entry points need a context (compar_init allocates) and grow a
// workspace on demand; this one needs neither.  Its only scratch memory — the
// split-K partial sums of the SIMT kernel — lives in a fixed file-scope
// device array, so the call allocates nothing.
//
// The paper has no counterpart of this entry point.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>
#include <string>

#include "common.h"

namespace {

// 16 MiB of split-K partial sums.  Every GPU that loads this library holds
// the array until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchBytes / sizeof(float)];

// Per-device set-up, once: the device check and the SM count.  The array's
// device address is looked up on every call instead (the host-side name of a
// __device__ array is not a device address): the lookup allocates nothing,
// and a context torn down and made again (cudaDeviceReset) may load the
// module, and with it the array, at another address.
using compar::kMaxDevices;
struct DeviceSetup {
  bool done = false;
  int num_sms = 0;
};
std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];

int setup_current_device(int* num_sms, float** scratch) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    compar::set_last_error_text("compar_gemm_simt_noalloc: no current CUDA device");
    return COMPAR_ERR_CUDA;
  }
  {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    DeviceSetup& d = g_setup[dev];
    if (!d.done) {
      int major = 0, minor = 0, sms = 0;
      if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        compar::set_last_error_text("compar_gemm_simt_noalloc: cannot query the device");
        return COMPAR_ERR_CUDA;
      }
      if (major != 10 || minor != 3) {
        compar::set_last_error_text("compar_gemm_simt_noalloc: built for sm_103 (B300) only");
        return COMPAR_ERR_UNSUPPORTED;
      }
      d.num_sms = sms;
      d.done = true;
    }
    *num_sms = d.num_sms;
  }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr) {
    compar::set_last_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
    return COMPAR_ERR_CUDA;
  }
  *scratch = static_cast<float*>(p);
  return COMPAR_OK;
}

}  // namespace

extern "C" int compar_gemm_simt_noalloc(int64_t m, int64_t n, int64_t k, float alpha,
                                        const float* A, const float* B, float beta, float* C,
                                        void* stream) {
  if (m < 0 || n < 0 || k < 0 || m > INT32_MAX || n > INT32_MAX || k > INT32_MAX)
    return COMPAR_ERR_INVALID;
  if ((m + 31) / 32 > 65535) return COMPAR_ERR_INVALID;
  if (m > 0 && n > 0 && C == nullptr) return COMPAR_ERR_INVALID;
  if (m > 0 && n > 0 && k > 0 && (A == nullptr || B == nullptr)) return COMPAR_ERR_INVALID;
  // a non-sticky error the caller left pending is not this call's launch
  // failing (clearing it allocates nothing)
  (void)cudaGetLastError();
  int num_sms = 0;
  float* scratch = nullptr;
  int rc = setup_current_device(&num_sms, &scratch);
  if (rc != COMPAR_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (m == 0 || n == 0) return COMPAR_OK;
  // A and B are not read when k == 0 or alpha == 0 (BLAS convention)
  if (k == 0 || alpha == 0.f) return compar::launch_scale_c(C, m, n, n, beta, s);
  compar::GemmCall c;
  c.m = m;
  c.n = n;
  c.k = k;
  c.lda = k;
  c.ldb = n;
  c.ldc = n;
  c.dtype = COMPAR_F32;
  c.A = A;
  c.B = B;
  c.C = C;
  c.alpha = alpha;
  c.beta = beta;
  size_t need = 0;
  rc = compar::launch_simt_scratch(c, scratch, kNoAllocScratchBytes, num_sms, s, &need);
  if (rc == COMPAR_ERR_INVALID) {
    char buf[256];
    snprintf(buf, sizeof(buf),
             "compar_gemm_simt_noalloc: %lldx%lldx%lld needs %zu bytes of split-K scratch; "
             "the limit is %zu bytes (16 MiB)",
             static_cast<long long>(m), static_cast<long long>(n), static_cast<long long>(k),
             need, kNoAllocScratchBytes);
    compar::set_last_error_text(buf);
  }
  return rc;
}
