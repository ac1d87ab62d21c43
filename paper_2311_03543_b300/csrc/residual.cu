// FP64 residual check on the GPU: the relative Frobenius error of a computed
// C against alpha * op_scale * A x B, evaluated in double precision on a
// seeded sample of rows.  It labels the error of recorded runs for the cost
// models (the selection must respect the accuracy a call asks for).
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "runtime.h"

namespace compar {
namespace {

__device__ __forceinline__ double elem(const void* base, int dtype, int64_t i) {
  if (dtype == COMPAR_F32) return static_cast<double>(static_cast<const float*>(base)[i]);
  if (dtype == COMPAR_BF16)
    return static_cast<double>(
        __uint_as_float(static_cast<uint32_t>(static_cast<const uint16_t*>(base)[i]) << 16));
  const __half_raw h = __nv_cvt_fp8_to_halfraw(
      static_cast<__nv_fp8_storage_t>(static_cast<const uint8_t*>(base)[i]), __NV_E4M3);
  return static_cast<double>(__half2float(__half(h)));
}

// Block r handles sampled row rows[r]; sums[2r] = sum (C - ref)^2,
// sums[2r+1] = sum ref^2 over that row.
__global__ void residual_kernel(int n, int k, int dtype, const void* __restrict__ A,
                                const void* __restrict__ B, const float* __restrict__ C,
                                double scale, const int64_t* __restrict__ rows,
                                double* __restrict__ sums) {
  const int64_t i = rows[blockIdx.x];
  double d2 = 0.0, r2 = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double acc = 0.0;
    for (int p = 0; p < k; ++p)
      acc = fma(elem(A, dtype, i * k + p), elem(B, dtype, static_cast<int64_t>(p) * n + j), acc);
    const double ref = scale * acc;
    const double diff = static_cast<double>(C[i * n + j]) - ref;
    d2 += diff * diff;
    r2 += ref * ref;
  }
  __shared__ double s0[32], s1[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    d2 += __shfl_xor_sync(0xffffffffu, d2, off);
    r2 += __shfl_xor_sync(0xffffffffu, r2, off);
  }
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  if (lane == 0) {
    s0[warp] = d2;
    s1[warp] = r2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x / 32); ++w) {
      a += s0[w];
      b += s1[w];
    }
    sums[2 * blockIdx.x] = a;
    sums[2 * blockIdx.x + 1] = b;
  }
}

uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace
}  // namespace compar

using namespace compar;

extern "C" int compar_residual_check(compar_ctx_t ctx, int64_t m, int64_t n, int64_t k,
                                     compar_dtype_t dtype, const void* A, const void* B,
                                     const float* C, float alpha, int nrows, uint64_t seed,
                                     double* rel_err, void* stream) {
  DeviceScope device_scope(ctx ? ctx->device : -1);
  if (!ctx || !rel_err || m <= 0 || n <= 0 || k <= 0 || nrows <= 0 || !A || !B || !C ||
      m > INT32_MAX || n > INT32_MAX || k > INT32_MAX ||
      (dtype != COMPAR_F32 && dtype != COMPAR_BF16 && dtype != COMPAR_F8E4M3))
    return COMPAR_ERR_INVALID;
  if (ctx->host_only) return COMPAR_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (int rc = refuse_capture(s, "compar_residual_check"); rc != COMPAR_OK)
    return rc;  // it reads its result back on the host
  // distinct sampled rows (all rows when nrows >= m)
  std::vector<int64_t> rows;
  if (nrows >= m) {
    for (int64_t i = 0; i < m; ++i) rows.push_back(i);
  } else {
    uint64_t st = seed;
    std::vector<char> used(static_cast<size_t>(m), 0);
    while (static_cast<int>(rows.size()) < nrows) {
      const int64_t i = static_cast<int64_t>(splitmix64(st) % static_cast<uint64_t>(m));
      if (!used[i]) {
        used[i] = 1;
        rows.push_back(i);
      }
    }
  }
  const int R = static_cast<int>(rows.size());
  int64_t* d_rows = nullptr;
  double* d_sums = nullptr;
  COMPAR_CUDA_TRY(cudaMallocAsync(&d_rows, R * sizeof(int64_t), s));
  COMPAR_CUDA_TRY(cudaMallocAsync(&d_sums, 2 * R * sizeof(double), s));
  COMPAR_CUDA_TRY(cudaMemcpyAsync(d_rows, rows.data(), R * sizeof(int64_t),
                                  cudaMemcpyHostToDevice, s));
  const double scale = static_cast<double>(alpha) *
                       (dtype == COMPAR_F8E4M3 ? static_cast<double>(ctx->scale_a) * ctx->scale_b
                                               : 1.0);
  residual_kernel<<<R, 256, 0, s>>>(static_cast<int>(n), static_cast<int>(k), dtype, A, B, C,
                                    scale, d_rows, d_sums);
  COMPAR_CUDA_TRY(cudaGetLastError());
  count_launch();
  std::vector<double> sums(2 * R);
  COMPAR_CUDA_TRY(cudaMemcpyAsync(sums.data(), d_sums, 2 * R * sizeof(double),
                                  cudaMemcpyDeviceToHost, s));
  COMPAR_CUDA_TRY(cudaFreeAsync(d_rows, s));
  COMPAR_CUDA_TRY(cudaFreeAsync(d_sums, s));
  COMPAR_CUDA_TRY(cudaStreamSynchronize(s));
  double num = 0, den = 0;
  for (int r = 0; r < R; ++r) {
    num += sums[2 * r];
    den += sums[2 * r + 1];
  }
  *rel_err = den > 0 ? std::sqrt(num / den) : (num > 0 ? INFINITY : 0.0);
  return COMPAR_OK;
}
