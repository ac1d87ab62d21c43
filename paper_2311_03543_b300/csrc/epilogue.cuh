// Epilogue stores shared by the tensor-core kernels: fragments of the
// accumulator as tcgen05.ld 16x256b delivers them (ptx.cuh), written to C
// with whole 32-byte sectors per row and instruction, or staged in shared
// memory and written by TMA bulk-tensor stores.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "ptx.cuh"

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

// TMA-store epilogue: each epilogue warp owns two 2 KB staging boxes (16
// rows x 32 float columns, 128-byte rows in the 128-byte swizzle: 16-byte
// chunk c of row r sits at chunk c ^ (r % 8)).  Stores the 16-row x
// 64-column fragment of store_frag's register layout as alpha * v, box by
// box: wait until the box's previous store has read it, write it (each
// float2 row pair lands in distinct banks: two wavefronts a store), make it
// visible to the async proxy, and lane 0 issues the bulk-tensor store.
// Boxes that start past the matrix are skipped; the tensor map clips the
// rest.  `nbox` counts the warp's boxes (buffer nbox & 1).
__device__ __forceinline__ void tma_store_frag(const CUtensorMap* tmC, uint8_t* stage,
                                               uint32_t& nbox, const float (&v)[32], int row0,
                                               int col0, int M, int N, float alpha, int lane) {
  if (row0 >= M) return;
  const int rq = lane >> 2;
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    const int cb0 = col0 + 32 * b;
    if (cb0 >= N) break;
    uint8_t* buf = stage + (nbox & 1u) * 2048u;
    if (lane == 0) dev::bulk_wait_read<1>();
    __syncwarp();
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int j = 4 * b + jj;
      const int c = 2 * jj + ((lane & 3) >> 1);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = rq + 8 * h;
        *reinterpret_cast<float2*>(buf + r * 128 + ((c ^ rq) << 4) + ((lane & 1) << 3)) =
            make_float2(alpha * v[4 * j + 2 * h], alpha * v[4 * j + 2 * h + 1]);
      }
    }
    dev::fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) {
      dev::tma_store_2d(tmC, buf, cb0, row0);
      dev::bulk_commit();
    }
    ++nbox;
  }
}

}  // namespace compar
