// FP32 FMA-pipe throughput microbenchmark: the denominator of the SIMT
// variants' roofline is measured on the device, not taken from a datasheet.
// Each thread runs 8 independent FMA chains in registers (enough
// instruction-level parallelism to keep the pipe busy); the result is written
// only when it equals a value it can never take, so nothing is optimised out.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "runtime.h"

namespace compar {
namespace {

__global__ void __launch_bounds__(256) ffma_kernel(int iters, float seed, float* sink) {
  float a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = seed + 0.001f * (threadIdx.x + j);
  const float x = 0.9999f, y = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int j = 0; j < 8; ++j) a[j] = fmaf(a[j], x, y);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  if (s == -12345.0f) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace compar

using namespace compar;

extern "C" int compar_peak_ffma(compar_ctx_t ctx, float* tflops, void* stream) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  if (!ctx || !tflops) return COMPAR_ERR_INVALID;
  if (ctx->host_only) return COMPAR_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* sink = nullptr;
  COMPAR_CUDA_TRY(cudaMallocAsync(&sink, 65536 * sizeof(float), s));
  const int blocks = ctx->num_sms * 8;  // 8 x 256 threads: full occupancy
  const int iters = 4096;
  cudaEvent_t e0, e1;
  COMPAR_CUDA_TRY(cudaEventCreate(&e0));
  COMPAR_CUDA_TRY(cudaEventCreate(&e1));
  ffma_kernel<<<blocks, 256, 0, s>>>(iters, 1.0f, sink);  // warm-up
  std::vector<float> t;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0, s);
    ffma_kernel<<<blocks, 256, 0, s>>>(iters, 1.0f + r, sink);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    t.push_back(ms);
  }
  count_launch(6);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  COMPAR_CUDA_TRY(cudaFreeAsync(sink, s));
  COMPAR_CUDA_TRY(cudaGetLastError());
  if (t.empty()) return COMPAR_ERR_CUDA;
  std::sort(t.begin(), t.end());
  const double flops = 2.0 * 8 * 16 * static_cast<double>(iters) * blocks * 256;
  *tflops = static_cast<float>(flops / (t[t.size() / 2] / 1e3) / 1e12);
  return COMPAR_OK;
}
