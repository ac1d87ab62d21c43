// Epilogue stores shared by the tensor-core kernels: fragments of the
// accumulator as tcgen05.ld 16x256b delivers them (ptx.cuh), written to C
// with whole 32-byte sectors per row and instruction.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace compar {

// Stores one 16-row x (8 J)-column fragment in the 16x256b.xJ register
// layout: v[4j + 2h + e] is row row0 + lane/4 + 8h, column
// col0 + 8j + 2(lane%4) + e.  C = alpha * v + beta * C (C not read when
// beta == 0); float2 stores when vec2 (even pitch, 8-byte base).  Rows >= M
// and columns >= N are not written.
template <int J>
__device__ __forceinline__ void store_frag(const float (&v)[4 * J], float* C, int64_t ldc, int M,
                                           int N, int row0, int col0, float alpha, float beta,
                                           bool vec2, int lane) {
  const int rq = lane >> 2, cq = 2 * (lane & 3);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int row = row0 + rq + 8 * h;
    if (row >= M) continue;
    float* crow = C + static_cast<int64_t>(row) * ldc;
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int col = col0 + 8 * j + cq;
      const float a = alpha * v[4 * j + 2 * h], b = alpha * v[4 * j + 2 * h + 1];
      if (vec2 && col + 1 < N) {
        float2* dst = reinterpret_cast<float2*>(crow + col);
        float2 o = make_float2(a, b);
        if (beta != 0.f) {
          const float2 old = *dst;
          o.x = fmaf(beta, old.x, o.x);
          o.y = fmaf(beta, old.y, o.y);
        }
        *dst = o;
      } else {
        if (col < N) crow[col] = beta != 0.f ? fmaf(beta, crow[col], a) : a;
        if (col + 1 < N) crow[col + 1] = beta != 0.f ? fmaf(beta, crow[col + 1], b) : b;
      }
    }
  }
}

}  // namespace compar
