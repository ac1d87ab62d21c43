// Operand pre-passes for the tensor-core variants: converting copies that
// write the K-major, 16-byte-pitched layouts TMA loads from.
//
//  * f32 -> bf16 (round to nearest even)                 (BF16 variant on f32 inputs)
//  * f32 -> (hi, lo) bf16 pair, hi = bf16(x), lo = bf16(x - hi)   (3xBF16 split)
//  * f32 -> (hi, mid, lo) bf16 triple, mid = bf16(x - hi),
//           lo = bf16(x - hi - mid)                         (6-product split)
//  * f32 -> (hi, lo) TF32 pair as float32, hi = tf32(x), lo = tf32(x - hi),
//           rounding to nearest, ties away from zero        (3xTF32 split)
//  * f32 -> E4M3 codes of x * s, s = 448 / amax(|x|), saturating   (FP8 variant)
//  * plain copy / transpose of f32, bf16 or fp8 elements
//
// B arrives row-major K x N; the tensor-core kernels read it as N x K
// (K-major), so its pre-pass transposes through a 32 x 32 shared-memory tile.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>

#include "common.h"
#include "grouped.h"
#include "ptx.cuh"

namespace compar {
namespace {

// One float32 value of a per-tensor FP8 quantisation: x * s rounded, then
// converted to E4M3 (round to nearest, saturating).  A non-finite x gives the
// E4M3 NaN code 0x7F, so an infinity stays non-finite (saturation would make
// it +-448) and stays local: the scale is taken over finite values only.
__device__ __forceinline__ __nv_fp8_storage_t e4m3_of(float x, float s) {
  return isfinite(x) ? __nv_cvt_float_to_fp8(__fmul_rn(x, s), __NV_SATFINITE, __NV_E4M3)
                     : static_cast<__nv_fp8_storage_t>(0x7F);
}

// |x| for the amax of a quantisation: non-finite values do not count.
__device__ __forceinline__ float finite_abs(float x) { return isfinite(x) ? fabsf(x) : 0.f; }


// Three-piece split; both residuals are exact in float32.
__device__ __forceinline__ void split3p(float x, __nv_bfloat16& h, __nv_bfloat16& m,
                                        __nv_bfloat16& l) {
  h = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(h);
  m = __float2bfloat16_rn(r1);
  l = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

// Nearest TF32 value (10 fraction bits, ties away from zero) of a finite
// float32, as a float32 with the low 13 bits clear: add half of the kept
// unit to the pattern and clear the dropped bits.
__device__ __forceinline__ float tf32_rna(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// Piece 2 of a split output: pieces are equally spaced, Y_lo = piece 1.
__device__ __forceinline__ __nv_bfloat16* piece2(void* Y, void* Ylo) {
  __nv_bfloat16* y = static_cast<__nv_bfloat16*>(Y);
  __nv_bfloat16* y1 = static_cast<__nv_bfloat16*>(Ylo);
  return y1 + (y1 - y);
}

// One element conversion for the float32-input kinds.
struct F32Out {
  int kind;
  float s;  // fp8 scale
};

__device__ __forceinline__ void store_converted(const F32Out& o, float x, void* Y, void* Ylo,
                                                int64_t idx) {
  switch (o.kind) {
    case PP_F32:
      static_cast<float*>(Y)[idx] = x;
      break;
    case PP_BF16:
      static_cast<__nv_bfloat16*>(Y)[idx] = __float2bfloat16_rn(x);
      break;
    case PP_SPLIT_BF16: {
      const __nv_bfloat16 hi = __float2bfloat16_rn(x);
      const float r = x - __bfloat162float(hi);
      static_cast<__nv_bfloat16*>(Y)[idx] = hi;
      static_cast<__nv_bfloat16*>(Ylo)[idx] = __float2bfloat16_rn(r);
      break;
    }
    case PP_SPLIT_BF16_3P: {
      __nv_bfloat16 h, m, l;
      split3p(x, h, m, l);
      static_cast<__nv_bfloat16*>(Y)[idx] = h;
      static_cast<__nv_bfloat16*>(Ylo)[idx] = m;
      piece2(Y, Ylo)[idx] = l;
      break;
    }
    case PP_SPLIT_TF32: {
      const float h = tf32_rna(x);
      static_cast<float*>(Y)[idx] = h;
      static_cast<float*>(Ylo)[idx] = tf32_rna(x - h);
      break;
    }
    case PP_E4M3:
      static_cast<__nv_fp8_storage_t*>(Y)[idx] = e4m3_of(x, o.s);
      break;
    default:
      break;
  }
}

// Non-transposing f32 conversion: Y[r][c] = f(X[r][c]).
__global__ void convert_rows_kernel(const float* __restrict__ X, int64_t rows, int64_t cols,
                                    int64_t ldx, void* __restrict__ Y, void* __restrict__ Ylo,
                                    int64_t ldy, int kind, const float* __restrict__ dscale) {
  F32Out o{kind, dscale ? *dscale : 1.f};
  // rows over blockIdx.y, columns over blockIdx.x / threads (no per-element
  // division)
  for (int64_t r = blockIdx.y; r < rows; r += gridDim.y)
    for (int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; c < cols;
         c += static_cast<int64_t>(gridDim.x) * blockDim.x)
      store_converted(o, X[r * ldx + c], Y, Ylo, r * ldy + c);
}

// Transposing f32 conversion: Y[c][r] = f(X[r][c]) through a 32x32 tile.
__global__ void convert_transpose_kernel(const float* __restrict__ X, int64_t rows, int64_t cols,
                                         int64_t ldx, void* __restrict__ Y,
                                         void* __restrict__ Ylo, int64_t ldy, int kind,
                                         const float* __restrict__ dscale) {
  __shared__ float tile[32][33];
  F32Out o{kind, dscale ? *dscale : 1.f};
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * 32;
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && c < cols) ? X[r * ldx + c] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t c = c0 + i, r = r0 + threadIdx.x;  // output row c, column r
    if (c < cols && r < rows) store_converted(o, tile[threadIdx.x][i], Y, Ylo, c * ldy + r);
  }
}

// ------------------------------------------------------------------ vectorised
// Eight consecutive float32 -> one packed group of the output kind.
__device__ __forceinline__ void store8(int kind, float s, const float (&x)[8], void* Y, void* Ylo,
                                      int64_t idx) {
  if (kind == PP_F32) {
    float4* y = reinterpret_cast<float4*>(static_cast<float*>(Y) + idx);
    y[0] = make_float4(x[0], x[1], x[2], x[3]);
    y[1] = make_float4(x[4], x[5], x[6], x[7]);
  } else if (kind == PP_SPLIT_TF32) {
    float h[8], l[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      h[q] = tf32_rna(x[q]);
      l[q] = tf32_rna(x[q] - h[q]);
    }
    float4* y = reinterpret_cast<float4*>(static_cast<float*>(Y) + idx);
    float4* z = reinterpret_cast<float4*>(static_cast<float*>(Ylo) + idx);
    y[0] = make_float4(h[0], h[1], h[2], h[3]);
    y[1] = make_float4(h[4], h[5], h[6], h[7]);
    z[0] = make_float4(l[0], l[1], l[2], l[3]);
    z[1] = make_float4(l[4], l[5], l[6], l[7]);
  } else if (kind == PP_SPLIT_BF16_3P) {
    uint32_t w[3][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      __nv_bfloat16 h0, m0, l0, h1, m1, l1;
      split3p(x[2 * q], h0, m0, l0);
      split3p(x[2 * q + 1], h1, m1, l1);
      w[0][q] = __bfloat16_as_ushort(h0) | (static_cast<uint32_t>(__bfloat16_as_ushort(h1)) << 16);
      w[1][q] = __bfloat16_as_ushort(m0) | (static_cast<uint32_t>(__bfloat16_as_ushort(m1)) << 16);
      w[2][q] = __bfloat16_as_ushort(l0) | (static_cast<uint32_t>(__bfloat16_as_ushort(l1)) << 16);
    }
    __nv_bfloat16* dst[3] = {static_cast<__nv_bfloat16*>(Y), static_cast<__nv_bfloat16*>(Ylo),
                             piece2(Y, Ylo)};
#pragma unroll
    for (int p = 0; p < 3; ++p)
      *reinterpret_cast<uint4*>(dst[p] + idx) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
  } else if (kind == PP_BF16 || kind == PP_SPLIT_BF16) {
    uint32_t hi[4], lo[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const __nv_bfloat16 h0 = __float2bfloat16_rn(x[2 * q]);
      const __nv_bfloat16 h1 = __float2bfloat16_rn(x[2 * q + 1]);
      hi[q] = static_cast<uint32_t>(__bfloat16_as_ushort(h0)) |
              (static_cast<uint32_t>(__bfloat16_as_ushort(h1)) << 16);
      if (kind == PP_SPLIT_BF16) {
        const __nv_bfloat16 l0 = __float2bfloat16_rn(x[2 * q] - __bfloat162float(h0));
        const __nv_bfloat16 l1 = __float2bfloat16_rn(x[2 * q + 1] - __bfloat162float(h1));
        lo[q] = static_cast<uint32_t>(__bfloat16_as_ushort(l0)) |
                (static_cast<uint32_t>(__bfloat16_as_ushort(l1)) << 16);
      }
    }
    *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(Y) + idx) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    if (kind == PP_SPLIT_BF16)
      *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(Ylo) + idx) =
          make_uint4(lo[0], lo[1], lo[2], lo[3]);
  } else {  // PP_E4M3
    uint32_t w[2] = {0u, 0u};
#pragma unroll
    for (int q = 0; q < 8; ++q)
      w[q / 4] |= static_cast<uint32_t>(e4m3_of(x[q], s)) << (8 * (q % 4));
    *reinterpret_cast<uint2*>(static_cast<uint8_t*>(Y) + idx) = make_uint2(w[0], w[1]);
  }
}

// Row-wise convert of float32 rows (8 elements per group, 16-byte aligned)
// of one or two matrices (rows of j0, then rows of j1): each thread takes
// kRowUnroll groups of one row, 256 groups apart, and issues all their
// loads before its stores, so that 128 bytes per thread are in flight; rows
// are dealt to the blocks of a resident-sized grid.  Launched
// programmatically: it waits for the stream's previous kernel first, and
// lets the next one (the GEMM) be scheduled at once.
constexpr int kRowUnroll = 4;
__global__ void convert_rows_vec8_kernel(const RowConvert j0, const RowConvert j1, int kind) {
  dev::griddep_wait();
  dev::griddep_launch_dependents();
  const float s0 = j0.dscale ? *j0.dscale : 1.f;
  const float s1 = (j1.rows > 0 && j1.dscale) ? *j1.dscale : 1.f;
  const int64_t rows_all = j0.rows + j1.rows;
  const int64_t span = static_cast<int64_t>(blockDim.x) * kRowUnroll;  // groups per block pass
  for (int64_t r_all = blockIdx.y; r_all < rows_all; r_all += gridDim.y) {
    const bool first = r_all < j0.rows;
    const int64_t r = first ? r_all : r_all - j0.rows;
    const int64_t groups = (first ? j0.cols : j1.cols) / 8;
    const float* xr = (first ? j0.X : j1.X) + r * (first ? j0.ldx : j1.ldx);
    void* Y = first ? j0.Y : j1.Y;
    void* Ylo = first ? j0.Y_lo : j1.Y_lo;
    const int64_t yoff = r * (first ? j0.ldy : j1.ldy);
    const float sc = first ? s0 : s1;
    for (int64_t g0 = blockIdx.x * span + threadIdx.x; g0 < groups;
         g0 += static_cast<int64_t>(gridDim.x) * span) {
      float4 a[kRowUnroll], b[kRowUnroll];
#pragma unroll
      for (int u = 0; u < kRowUnroll; ++u) {
        const int64_t gi = g0 + u * static_cast<int64_t>(blockDim.x);
        if (gi < groups) {
          const float4* src = reinterpret_cast<const float4*>(xr + gi * 8);
          a[u] = __ldg(src);
          b[u] = __ldg(src + 1);
        }
      }
#pragma unroll
      for (int u = 0; u < kRowUnroll; ++u) {
        const int64_t gi = g0 + u * static_cast<int64_t>(blockDim.x);
        if (gi < groups) {
          const float x[8] = {a[u].x, a[u].y, a[u].z, a[u].w, b[u].x, b[u].y, b[u].z, b[u].w};
          store8(kind, sc, x, Y, Ylo, yoff + gi * 8);
        }
      }
    }
  }
}

// The vectorised row kernel's rules for one matrix.
bool rows_vec8_ok(const RowConvert& j) {
  const uintptr_t xa = reinterpret_cast<uintptr_t>(j.X), ya = reinterpret_cast<uintptr_t>(j.Y),
                  la = reinterpret_cast<uintptr_t>(j.Y_lo);
  return j.cols % 8 == 0 && j.ldx % 4 == 0 && xa % 16 == 0 && j.ldy % 8 == 0 && ya % 16 == 0 &&
         la % 16 == 0;
}

// One launch of the row kernel over j0 and j1 (j1.rows may be 0): blocks
// across a row cover it in passes of 256 x kRowUnroll groups; rows are dealt
// to about eight resident blocks per SM.
int launch_rows_vec8(const RowConvert& j0, const RowConvert& j1, int kind, int num_sms,
                     cudaStream_t s) {
  const int64_t groups = std::max(j0.cols, j1.rows > 0 ? j1.cols : 0) / 8;
  const int64_t rows = j0.rows + j1.rows;
  const int64_t bx = std::max<int64_t>(
      1, std::min<int64_t>((groups + 256 * kRowUnroll - 1) / (256 * kRowUnroll), 64));
  const int64_t by = std::max<int64_t>(1, std::min<int64_t>(rows, std::min<int64_t>(
                                              65535, (8 * static_cast<int64_t>(num_sms) + bx - 1) / bx)));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(bx), static_cast<unsigned>(by));
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  COMPAR_CUDA_TRY(cudaLaunchKernelEx(&cfg, convert_rows_vec8_kernel, j0, j1, kind));
  count_launch();
  return COMPAR_OK;
}

// Transposing convert through a 64 x 64 tile: float2 loads, each thread
// stores two consecutive outputs (bf16 pairs, float2, or two bytes).
__global__ void convert_transpose64_kernel(const float* __restrict__ X, int64_t rows, int64_t cols,
                                           int64_t ldx, void* __restrict__ Y,
                                           void* __restrict__ Ylo, int64_t ldy, int kind,
                                           const float* __restrict__ dscale) {
  __shared__ float tile[64][65];
  // when launched programmatically, the stream's previous kernel has
  // completed past this point
  dev::griddep_wait();
  dev::griddep_launch_dependents();
  const float s = dscale ? *dscale : 1.f;
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * 64;
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * 64;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int i = ty; i < 64; i += 8) {
    const int64_t r = r0 + i, c = c0 + 2 * tx;
    float2 v = make_float2(0.f, 0.f);
    if (r < rows) {
      if (c + 1 < cols) v = __ldg(reinterpret_cast<const float2*>(X + r * ldx + c));
      else if (c < cols) v.x = X[r * ldx + c];
    }
    tile[i][2 * tx] = v.x;
    tile[i][2 * tx + 1] = v.y;
  }
  __syncthreads();
  for (int j = ty; j < 64; j += 8) {  // output row c0 + j holds input column c0 + j
    const int64_t orow = c0 + j;
    const int64_t ocol = r0 + 2 * tx;
    if (orow >= cols || ocol >= rows) continue;
    const float x0 = tile[2 * tx][j], x1 = tile[2 * tx + 1][j];
    const int64_t idx = orow * ldy + ocol;
    if (ocol + 1 < rows) {
      if (kind == PP_F32) {
        *reinterpret_cast<float2*>(static_cast<float*>(Y) + idx) = make_float2(x0, x1);
      } else if (kind == PP_SPLIT_TF32) {
        const float h0 = tf32_rna(x0), h1 = tf32_rna(x1);
        *reinterpret_cast<float2*>(static_cast<float*>(Y) + idx) = make_float2(h0, h1);
        *reinterpret_cast<float2*>(static_cast<float*>(Ylo) + idx) =
            make_float2(tf32_rna(x0 - h0), tf32_rna(x1 - h1));
      } else if (kind == PP_BF16 || kind == PP_SPLIT_BF16) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
        *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(Y) + idx) =
            __halves2bfloat162(h0, h1);
        if (kind == PP_SPLIT_BF16)
          *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(Ylo) + idx) =
              __halves2bfloat162(__float2bfloat16_rn(x0 - __bfloat162float(h0)),
                                 __float2bfloat16_rn(x1 - __bfloat162float(h1)));
      } else if (kind == PP_SPLIT_BF16_3P) {
        __nv_bfloat16 h0, m0, l0, h1, m1, l1;
        split3p(x0, h0, m0, l0);
        split3p(x1, h1, m1, l1);
        *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(Y) + idx) =
            __halves2bfloat162(h0, h1);
        *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(Ylo) + idx) =
            __halves2bfloat162(m0, m1);
        *reinterpret_cast<__nv_bfloat162*>(piece2(Y, Ylo) + idx) = __halves2bfloat162(l0, l1);
      } else {
        uint8_t* y = static_cast<uint8_t*>(Y) + idx;
        y[0] = e4m3_of(x0, s);
        y[1] = e4m3_of(x1, s);
      }
    } else {
      store_converted(F32Out{kind, s}, x0, Y, Ylo, idx);
    }
  }
}

// Element-type-preserving copy (optionally transposing) for 1/2/4-byte types.
template <typename T>
__global__ void copy_kernel(const T* __restrict__ X, int64_t rows, int64_t cols, int64_t ldx,
                            T* __restrict__ Y, int64_t ldy) {
  for (int64_t r = blockIdx.y; r < rows; r += gridDim.y)
    for (int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; c < cols;
         c += static_cast<int64_t>(gridDim.x) * blockDim.x)
      Y[r * ldy + c] = X[r * ldx + c];
}

template <typename T>
__global__ void transpose_kernel(const T* __restrict__ X, int64_t rows, int64_t cols, int64_t ldx,
                                 T* __restrict__ Y, int64_t ldy) {
  __shared__ T tile[32][33];
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * 32;
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[i][threadIdx.x] = X[r * ldx + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < rows) Y[c * ldy + r] = tile[threadIdx.x][i];
  }
}

// amax(|X|) and amax(|Y|) in one launch, as float bits (non-negative floats
// order like their bit patterns): warp w of the grid takes rows w, w + warps,
// ... of the rows of X followed by those of Y, reading each row with 16-byte
// loads when its start is 16-byte aligned.
__device__ __forceinline__ float row_amax(const float* __restrict__ row, int64_t cols, int lane) {
  float m = 0.f;
  int64_t c = 0;
  if ((reinterpret_cast<uintptr_t>(row) & 15) == 0) {
    const float4* r4 = reinterpret_cast<const float4*>(row);
    const int64_t n4 = cols / 4;
    for (int64_t i = lane; i < n4; i += 32) {
      const float4 v = __ldg(r4 + i);
      m = fmaxf(m, fmaxf(fmaxf(finite_abs(v.x), finite_abs(v.y)),
                         fmaxf(finite_abs(v.z), finite_abs(v.w))));
    }
    c = n4 * 4;
  }
  for (int64_t i = c + lane; i < cols; i += 32) m = fmaxf(m, finite_abs(__ldg(row + i)));
  return m;
}

// amax(|X|) and amax(|Y|) of one block's rows: block b writes its maxima to
// out[2 b], out[2 b + 1] (no atomics, so nothing needs clearing first).
// Launched programmatically: it waits for the stream's previous kernel.
__global__ void amax2_kernel(const float* __restrict__ X, int64_t xr, int64_t xc, int64_t ldx,
                             const float* __restrict__ Y, int64_t yr, int64_t yc, int64_t ldy,
                             float* __restrict__ out) {
  dev::griddep_wait();
  dev::griddep_launch_dependents();
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  const int64_t nwarps = static_cast<int64_t>(gridDim.x) * (blockDim.x / 32);
  float mx = 0.f, my = 0.f;
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * (blockDim.x / 32) + warp; r < xr + yr;
       r += nwarps) {
    if (r < xr) mx = fmaxf(mx, row_amax(X + r * ldx, xc, lane));
    else my = fmaxf(my, row_amax(Y + (r - xr) * ldy, yc, lane));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, off));
  }
  __shared__ float wx[32], wy[32];
  if (lane == 0) {
    wx[warp] = mx;
    wy[warp] = my;
  }
  __syncthreads();
  if (warp == 0) {
    const bool in = lane < static_cast<int>(blockDim.x / 32);
    mx = in ? wx[lane] : 0.f;
    my = in ? wy[lane] : 0.f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
      my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, off));
    }
    if (lane == 0) {
      out[2 * blockIdx.x] = mx;
      out[2 * blockIdx.x + 1] = my;
    }
  }
}

// The per-block maxima of amax2_kernel (nblocks pairs) reduced to the two
// amaxes, then {s_x, 1/s_x, s_y, 1/s_y} with s = min(448 / amax, 2^126) (1
// when amax is 0), jointly reduced by powers of two so that 1 / (s_x s_y)
// stays a normal float32.  One block of 256 threads; launched programmatically.
__global__ void fp8_scales_kernel(const float* __restrict__ block_max, int nblocks,
                                  float* __restrict__ out) {
  dev::griddep_wait();
  dev::griddep_launch_dependents();
  float mx = 0.f, my = 0.f;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    mx = fmaxf(mx, block_max[2 * b]);
    my = fmaxf(my, block_max[2 * b + 1]);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, off));
  }
  __shared__ float wx[8], wy[8];
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  if (lane == 0) {
    wx[warp] = mx;
    wy[warp] = my;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float ax = 0.f, ay = 0.f;
    for (int w = 0; w < static_cast<int>(blockDim.x / 32); ++w) {
      ax = fmaxf(ax, wx[w]);
      ay = fmaxf(ay, wy[w]);
    }
    // Each scale is capped at 2^126 (448 / amax overflows float32 for amax <
    // 448 / FLT_MAX).  The dequantisation 1 / (s_x s_y) multiplies into
    // alpha, so it must stay a normal float32: when the scales' exponents
    // add up past 124, that many powers of two come off them, split evenly
    // (exact, so the product stays below 2^126).
    float sx = fminf(ax > 0.f ? __fdiv_rn(448.0f, ax) : 1.0f, 0x1p126f);
    float sy = fminf(ay > 0.f ? __fdiv_rn(448.0f, ay) : 1.0f, 0x1p126f);
    const int d = ilogbf(sx) + ilogbf(sy) - 124;
    if (d > 0) {
      sx = ldexpf(sx, -((d + 1) / 2));
      sy = ldexpf(sy, -(d / 2));
    }
    out[0] = sx;
    out[1] = __fdiv_rn(1.0f, sx);
    out[2] = sy;
    out[3] = __fdiv_rn(1.0f, sy);
  }
}

// ------------------------------------------------------------------ grouped

// Every operand re-layout of a batch in one launch.  The 64 x 64 tiles of
// all jobs form one list (job j owns [tile_start, tile_start + tiles)); each
// block converts one contiguous run of that list, so big and small jobs
// spread evenly over the grid and a block changes job only at a boundary.
//
// Per tile the work is specialised on (input type, output kind, transpose):
// no per-element switch, 4-wide global loads when the job's rows are 16-byte
// aligned, and stores of two (transposed) or four (row-wise) consecutive
// outputs per thread, so a warp writes whole 128-byte lines.

// Output of 1, 2 or 4 consecutive elements of one piece row.
template <int KIND>
struct PieceOut;
template <>
struct PieceOut<PP_F32> {
  static __device__ __forceinline__ void put2(void* Y, void*, int64_t i, float a, float b) {
    *reinterpret_cast<float2*>(static_cast<float*>(Y) + i) = make_float2(a, b);
  }
  static __device__ __forceinline__ void put4(void* Y, void*, int64_t i, float4 v) {
    *reinterpret_cast<float4*>(static_cast<float*>(Y) + i) = v;
  }
  static __device__ __forceinline__ void put1(void* Y, void*, int64_t i, float a) {
    static_cast<float*>(Y)[i] = a;
  }
};
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  return static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(a))) |
         (static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(b))) << 16);
}
template <>
struct PieceOut<PP_BF16> {
  static __device__ __forceinline__ void put2(void* Y, void*, int64_t i, float a, float b) {
    *reinterpret_cast<uint32_t*>(static_cast<__nv_bfloat16*>(Y) + i) = pack_bf16(a, b);
  }
  static __device__ __forceinline__ void put4(void* Y, void*, int64_t i, float4 v) {
    *reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(Y) + i) =
        make_uint2(pack_bf16(v.x, v.y), pack_bf16(v.z, v.w));
  }
  static __device__ __forceinline__ void put1(void* Y, void*, int64_t i, float a) {
    static_cast<__nv_bfloat16*>(Y)[i] = __float2bfloat16_rn(a);
  }
};
template <>
struct PieceOut<PP_SPLIT_BF16> {
  static __device__ __forceinline__ float lo(float x) {
    return x - __bfloat162float(__float2bfloat16_rn(x));
  }
  static __device__ __forceinline__ void put2(void* Y, void* L, int64_t i, float a, float b) {
    *reinterpret_cast<uint32_t*>(static_cast<__nv_bfloat16*>(Y) + i) = pack_bf16(a, b);
    *reinterpret_cast<uint32_t*>(static_cast<__nv_bfloat16*>(L) + i) = pack_bf16(lo(a), lo(b));
  }
  static __device__ __forceinline__ void put4(void* Y, void* L, int64_t i, float4 v) {
    *reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(Y) + i) =
        make_uint2(pack_bf16(v.x, v.y), pack_bf16(v.z, v.w));
    *reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(L) + i) =
        make_uint2(pack_bf16(lo(v.x), lo(v.y)), pack_bf16(lo(v.z), lo(v.w)));
  }
  static __device__ __forceinline__ void put1(void* Y, void* L, int64_t i, float a) {
    static_cast<__nv_bfloat16*>(Y)[i] = __float2bfloat16_rn(a);
    static_cast<__nv_bfloat16*>(L)[i] = __float2bfloat16_rn(lo(a));
  }
};

// Four consecutive inputs as float (vector load when `vec`).
template <typename In>
__device__ __forceinline__ float4 load4(const In* p, bool vec, int n_valid);
template <>
__device__ __forceinline__ float4 load4<float>(const float* p, bool vec, int n_valid) {
  if (vec && n_valid >= 4) return __ldg(reinterpret_cast<const float4*>(p));
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (n_valid > 0) v.x = __ldg(p);
  if (n_valid > 1) v.y = __ldg(p + 1);
  if (n_valid > 2) v.z = __ldg(p + 2);
  if (n_valid > 3) v.w = __ldg(p + 3);
  return v;
}
template <>
__device__ __forceinline__ float4 load4<__nv_bfloat16>(const __nv_bfloat16* p, bool vec,
                                                       int n_valid) {
  if (vec && n_valid >= 4) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xFFFF0000u),
                       __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xFFFF0000u));
  }
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (n_valid > 0) v.x = __bfloat162float(p[0]);
  if (n_valid > 1) v.y = __bfloat162float(p[1]);
  if (n_valid > 2) v.z = __bfloat162float(p[2]);
  if (n_valid > 3) v.w = __bfloat162float(p[3]);
  return v;
}

// Row-wise job: Y[r][c] = f(X[r][c]); thread = 4 consecutive columns of 4
// rows, all four loads issued before the first store.
template <typename In, int KIND>
__device__ __forceinline__ void tile_rows(const PrepassJob& J, int64_t r0, int64_t c0) {
  const In* X = static_cast<const In*>(J.src);
  const bool vec = J.vec != 0;
  float4 vq[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int idx = threadIdx.x + 256 * q;  // 64 rows x 16 groups of 4
    const int64_t r = r0 + (idx >> 4);
    const int64_t c = c0 + 4 * (idx & 15);
    if (r >= J.rows || c >= J.cols) continue;
    const int64_t rem = J.cols - c;
    vq[q] = load4<In>(X + r * J.ld_src + c, vec, rem >= 4 ? 4 : static_cast<int>(rem));
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int idx = threadIdx.x + 256 * q;
    const int64_t r = r0 + (idx >> 4);
    const int64_t c = c0 + 4 * (idx & 15);
    if (r >= J.rows || c >= J.cols) continue;
    const int64_t rem = J.cols - c;
    const int n_valid = rem >= 4 ? 4 : static_cast<int>(rem);
    const float4 v = vq[q];
    const int64_t o = r * J.ld_dst + c;
    if (n_valid == 4) {  // outputs rows have pitch ldk (a multiple of 16): aligned
      PieceOut<KIND>::put4(J.dst, J.dst_lo, o, v);
    } else {  // ragged right edge: 1 to 3 columns
      PieceOut<KIND>::put1(J.dst, J.dst_lo, o, v.x);
      if (n_valid > 1) PieceOut<KIND>::put1(J.dst, J.dst_lo, o + 1, v.y);
      if (n_valid > 2) PieceOut<KIND>::put1(J.dst, J.dst_lo, o + 2, v.z);
    }
  }
}

// Transposing job: Y[c][r] = f(X[r][c]) through shared memory.  Loads: a
// thread reads 4 consecutive columns of a row; stores: a warp writes 64
// consecutive r of one output row, two per thread.
template <typename In, int KIND>
__device__ __forceinline__ void tile_transpose(const PrepassJob& J, int64_t r0, int64_t c0,
                                               float (*tile)[65]) {
  const In* X = static_cast<const In*>(J.src);
  const bool vec = J.vec != 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int idx = threadIdx.x + 256 * q;
    const int lr = idx >> 4, lc = 4 * (idx & 15);
    const int64_t r = r0 + lr, c = c0 + lc;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < J.rows && c < J.cols) {
      const int64_t rem = J.cols - c;
      v = load4<In>(X + r * J.ld_src + c, vec, rem >= 4 ? 4 : static_cast<int>(rem));
    }
    tile[lr][lc] = v.x;
    tile[lr][lc + 1] = v.y;
    tile[lr][lc + 2] = v.z;
    tile[lr][lc + 3] = v.w;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lr = 2 * lane;
  const int64_t r = r0 + lr;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int lc = warp * 8 + i;  // output row c0 + lc
    const int64_t c = c0 + lc;
    if (c >= J.cols || r >= J.rows) continue;
    const float a = tile[lr][lc], b = tile[lr + 1][lc];
    const int64_t o = c * J.ld_dst + r;
    if (r + 1 < J.rows) PieceOut<KIND>::put2(J.dst, J.dst_lo, o, a, b);
    else PieceOut<KIND>::put1(J.dst, J.dst_lo, o, a);
  }
  __syncthreads();
}

// kTranspose: the batch has transposing jobs (the 64 x 64 staging tile in
// shared memory); without them the kernel uses no shared memory, so its
// blocks fit beside a grouped GEMM CTA on the same SM.
template <bool kTranspose>
__global__ void __launch_bounds__(256, 4) grouped_prepass_kernel(const PrepassJob* __restrict__ jobs,
                                                              int njobs, int total_tiles) {
  __shared__ float tile[kTranspose ? 64 : 1][65];
  const int per = (total_tiles + gridDim.x - 1) / gridDim.x;
  const int t_begin = blockIdx.x * per;
  const int t_end = min(total_tiles, t_begin + per);
  if (t_begin >= t_end) return;
  // the last job starting at or before t_begin (jobs are in tile order)
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&jobs[mid].tile_start) <= t_begin) lo = mid;
    else hi = mid - 1;
  }
  int j = lo;
  PrepassJob J = jobs[j];
  for (int t = t_begin; t < t_end; ++t) {
    while (t >= J.tile_start + J.tiles && j + 1 < njobs) J = jobs[++j];
    const int lt = t - J.tile_start;
    const int64_t r0 = static_cast<int64_t>(lt / J.tiles_c) * 64;
    const int64_t c0 = static_cast<int64_t>(lt % J.tiles_c) * 64;
    const bool f32 = J.in_type == COMPAR_F32;
    if (kTranspose && J.transpose) {
      if constexpr (kTranspose) {
        if (!f32) tile_transpose<__nv_bfloat16, PP_BF16>(J, r0, c0, tile);
        else if (J.out_kind == PP_SPLIT_BF16) tile_transpose<float, PP_SPLIT_BF16>(J, r0, c0, tile);
        else tile_transpose<float, PP_F32>(J, r0, c0, tile);
      }
    } else {
      if (!f32) tile_rows<__nv_bfloat16, PP_BF16>(J, r0, c0);
      else if (J.out_kind == PP_SPLIT_BF16) tile_rows<float, PP_SPLIT_BF16>(J, r0, c0);
      else tile_rows<float, PP_F32>(J, r0, c0);
    }
  }
}

}  // namespace

int launch_grouped_prepass(const PrepassJob* d_jobs, int njobs, int total_tiles, int num_sms,
                           bool transpose, cudaStream_t s) {
  if (njobs <= 0 || total_tiles <= 0) return COMPAR_OK;
  // one full wave of resident blocks
  // (queried once per device; threads driving other contexts may race to
  // fill it, with the same value)
  static std::atomic<int> resident[kMaxDevices][2] = {};
  const int d = current_device_index();
  if (d < 0) {
    set_last_error_text("grouped pre-pass: no usable current device");
    return COMPAR_ERR_CUDA;
  }
  int r = resident[d][transpose ? 1 : 0].load(std::memory_order_relaxed);
  if (r == 0) {
    int n = 0;
    COMPAR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &n, transpose ? grouped_prepass_kernel<true> : grouped_prepass_kernel<false>, 256, 0));
    r = std::max(n, 1);
    resident[d][transpose ? 1 : 0].store(r, std::memory_order_relaxed);
  }
  const int grid = static_cast<int>(std::min<int64_t>(total_tiles, static_cast<int64_t>(num_sms) * r));
  if (transpose)
    grouped_prepass_kernel<true><<<grid, 256, 0, s>>>(d_jobs, njobs, total_tiles);
  else
    grouped_prepass_kernel<false><<<grid, 256, 0, s>>>(d_jobs, njobs, total_tiles);
  COMPAR_CUDA_TRY(cudaGetLastError());
  count_launch();
  return COMPAR_OK;
}

namespace {
// Launch configuration with programmatic stream serialisation (the kernel
// waits for the stream's previous kernel itself); attr: one attribute.
cudaLaunchConfig_t programmatic_config(dim3 grid, dim3 block, cudaStream_t s,
                                       cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}
}  // namespace

int prepass_convert(const void* X, compar_dtype_t in_t, int64_t rows, int64_t cols, int64_t ldx,
                    void* Y, int out_kind, int64_t ldy, bool transpose, void* Y_lo,
                    const float* dscale, int num_sms, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return COMPAR_OK;
  const dim3 tb(32, 8);
  const dim3 tg(static_cast<unsigned>((cols + 31) / 32), static_cast<unsigned>((rows + 31) / 32));
  // row-wise kernels: 256 columns per block, rows over y (grid-stride past 65535)
  const dim3 rg(static_cast<unsigned>(std::min<int64_t>((cols + 255) / 256, 64)),
                static_cast<unsigned>(std::min<int64_t>(rows, 65535)));
  // float32 sources with aligned rows take the vectorised kernels
  if (in_t == COMPAR_F32 && (out_kind != PP_COPY || transpose)) {
    const int kind = out_kind == PP_COPY ? PP_F32 : out_kind;
    const float* Xf = static_cast<const float*>(X);
    const uintptr_t xa = reinterpret_cast<uintptr_t>(X), ya = reinterpret_cast<uintptr_t>(Y),
                    la = reinterpret_cast<uintptr_t>(Y_lo);
    if (transpose && cols % 2 == 0 && ldx % 2 == 0 && xa % 8 == 0 && ldy % 2 == 0 &&
        ya % 8 == 0 && la % 8 == 0 && rows < (int64_t(65535) * 64)) {
      const dim3 g64(static_cast<unsigned>((cols + 63) / 64), static_cast<unsigned>((rows + 63) / 64));
      // a normal launch (programmatic measured 2 us slower on the 6-product
      // split at 1024^3); the kernel's wait then returns at once
      convert_transpose64_kernel<<<g64, tb, 0, s>>>(Xf, rows, cols, ldx, Y, Y_lo, ldy, kind,
                                                   dscale);
      COMPAR_CUDA_TRY(cudaGetLastError());
      count_launch();
      return COMPAR_OK;
    }
    const RowConvert j{Xf, rows, cols, ldx, Y, Y_lo, ldy, dscale};
    if (!transpose && rows_vec8_ok(j)) {
      const RowConvert none{nullptr, 0, 0, 0, nullptr, nullptr, 0, nullptr};
      return launch_rows_vec8(j, none, kind, num_sms, s);
    }
  }
  if (out_kind == PP_COPY) {
    if (in_t == COMPAR_F32) {
      if (transpose)
        transpose_kernel<float><<<tg, tb, 0, s>>>(static_cast<const float*>(X), rows, cols, ldx,
                                                  static_cast<float*>(Y), ldy);
      else
        copy_kernel<float><<<rg, 256, 0, s>>>(
            static_cast<const float*>(X), rows, cols, ldx, static_cast<float*>(Y), ldy);
    } else if (in_t == COMPAR_BF16) {
      if (transpose)
        transpose_kernel<uint16_t><<<tg, tb, 0, s>>>(static_cast<const uint16_t*>(X), rows, cols,
                                                     ldx, static_cast<uint16_t*>(Y), ldy);
      else
        copy_kernel<uint16_t><<<rg, 256, 0, s>>>(
            static_cast<const uint16_t*>(X), rows, cols, ldx, static_cast<uint16_t*>(Y), ldy);
    } else {
      if (transpose)
        transpose_kernel<uint8_t><<<tg, tb, 0, s>>>(static_cast<const uint8_t*>(X), rows, cols,
                                                    ldx, static_cast<uint8_t*>(Y), ldy);
      else
        copy_kernel<uint8_t><<<rg, 256, 0, s>>>(
            static_cast<const uint8_t*>(X), rows, cols, ldx, static_cast<uint8_t*>(Y), ldy);
    }
  } else {
    if (in_t != COMPAR_F32) return COMPAR_ERR_INVALID;
    const float* Xf = static_cast<const float*>(X);
    if (transpose)
      convert_transpose_kernel<<<tg, tb, 0, s>>>(Xf, rows, cols, ldx, Y, Y_lo, ldy, out_kind,
                                                 dscale);
    else
      convert_rows_kernel<<<rg, 256, 0, s>>>(Xf, rows, cols, ldx, Y, Y_lo, ldy, out_kind, dscale);
  }
  COMPAR_CUDA_TRY(cudaGetLastError());
  count_launch();
  return COMPAR_OK;
}

int prepass_convert_rows2(const RowConvert& a, const RowConvert& b, int out_kind, int num_sms,
                          cudaStream_t s) {
  if (out_kind == PP_COPY || !rows_vec8_ok(a) || !rows_vec8_ok(b)) return COMPAR_ERR_UNSUPPORTED;
  if (a.rows <= 0 || a.cols <= 0 || b.rows <= 0 || b.cols <= 0) return COMPAR_ERR_UNSUPPORTED;
  return launch_rows_vec8(a, b, out_kind, num_sms, s);
}


int prepass_amax2(const float* X, int64_t xr, int64_t xc, int64_t ldx, const float* Y, int64_t yr,
                  int64_t yc, int64_t ldy, float* d_block_max, int max_blocks, int num_sms,
                  int* nblocks, cudaStream_t s) {
  *nblocks = 0;
  const int64_t rows = (xc > 0 ? xr : 0) + (yc > 0 ? yr : 0);
  if (rows <= 0) return COMPAR_OK;
  // 8 warps per block, one row per warp at a time; up to 8 blocks per SM
  const int grid = static_cast<int>(
      std::min<int64_t>(std::min<int64_t>((rows + 7) / 8, 8LL * num_sms), max_blocks));
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = programmatic_config(dim3(grid), dim3(256), s, attr);
  COMPAR_CUDA_TRY(cudaLaunchKernelEx(&cfg, amax2_kernel, X, xc > 0 ? xr : 0, xc, ldx, Y,
                                     yc > 0 ? yr : 0, yc, ldy, d_block_max));
  count_launch();
  *nblocks = grid;
  return COMPAR_OK;
}

int prepass_fp8_scales(const float* d_block_max, int nblocks, float* d_out, cudaStream_t s) {
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = programmatic_config(dim3(1), dim3(256), s, attr);
  COMPAR_CUDA_TRY(cudaLaunchKernelEx(&cfg, fp8_scales_kernel, d_block_max, nblocks, d_out));
  count_launch();
  return COMPAR_OK;
}

}  // namespace compar
