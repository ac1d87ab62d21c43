// Thermal 2-D stencil (the hotspot-like second component behind the same
// runtime; the paper evaluates Rodinia's Hotspot with CUDA and OpenMP
// variants, Table 2).  One explicit step of the 2-D heat equation with a
// power source and a leak to ambient, insulated grid edge:
//
//   T'[i][j] = T[i][j] + c * ( P[i][j] + (T[i-1][j] + T[i+1][j] - 2T[i][j]) * gy
//                                      + (T[i][j-1] + T[i][j+1] - 2T[i][j]) * gx
//                                      + (amb - T[i][j]) * gz )
//
// with a neighbour outside the grid replaced by the cell itself.  Every
// variant evaluates this with the same rounded operations (cell_update), so
// all variants give bit-identical grids.
//
//   NAIVE : one thread per cell, one launch per step, neighbours from global
//           memory (through L1/L2); ping-pong between two device grids.
//   TILED : temporal blocking: a CTA loads the 128 x 80 region around its
//           112 x 64 tile into shared memory and advances it up to 8 steps
//           there, writing the centre; ceil(steps / 8) launches.
//   TMA   : TILED with the region loaded by one TMA box into shared memory,
//           completion on an mbarrier (bounded wait).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "common.h"
#include "ptx.cuh"

namespace compar {
namespace {

struct Coef {
  float c, gx, gy, gz, amb;
};

// The step of one cell with a fixed order of rounded operations.
__device__ __forceinline__ float cell_update(float t, float n, float s, float w, float e, float p,
                                             const Coef& k) {
  const float two_t = __fmul_rn(2.f, t);
  const float dy = __fsub_rn(__fadd_rn(n, s), two_t);
  const float dx = __fsub_rn(__fadd_rn(w, e), two_t);
  float f = __fmaf_rn(dy, k.gy, p);
  f = __fmaf_rn(dx, k.gx, f);
  f = __fmaf_rn(__fsub_rn(k.amb, t), k.gz, f);
  return __fmaf_rn(k.c, f, t);
}

// The same step for two cells with packed FP32 pair instructions: every
// element is rounded exactly as in cell_update (x - y is x + (-y), the
// product by -2 is exact, and amb - t is the single rounding of
// fma(t, -1, amb)), so the results are bit-identical at half the
// instruction count.
struct Coef2 {
  float2 c, gx, gy, gz, amb;
};

__device__ __forceinline__ float2 cell_update2(float2 t, float2 n, float2 s, float2 w, float2 e,
                                               float2 p, const Coef2& k) {
  const float2 m2t = __fmul2_rn(t, make_float2(-2.f, -2.f));
  const float2 dy = __fadd2_rn(__fadd2_rn(n, s), m2t);
  const float2 dx = __fadd2_rn(__fadd2_rn(w, e), m2t);
  float2 f = __ffma2_rn(dy, k.gy, p);
  f = __ffma2_rn(dx, k.gx, f);
  f = __ffma2_rn(__ffma2_rn(t, make_float2(-1.f, -1.f), k.amb), k.gz, f);
  return __ffma2_rn(k.c, f, t);
}

// ------------------------------------------------------------------ NAIVE
__global__ void stencil_naive_kernel(const float* __restrict__ T, const float* __restrict__ P,
                                     float* __restrict__ out, int rows, int cols, Coef k) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= rows || j >= cols) return;
  const int64_t idx = static_cast<int64_t>(i) * cols + j;
  const float t = T[idx];
  const float n = i > 0 ? T[idx - cols] : t;
  const float s = i < rows - 1 ? T[idx + cols] : t;
  const float w = j > 0 ? T[idx - 1] : t;
  const float e = j < cols - 1 ? T[idx + 1] : t;
  out[idx] = cell_update(t, n, s, w, e, P[idx], k);
}

// ------------------------------------------------------------------ TILED / TMA
// A CTA owns a 112 x 64 output tile (columns x rows) and advances the
// 128 x 80 region around it (8-cell halo) up to 8 steps in shared memory.
// The region sits in an 82 x 136 buffer: one pad row above and below, 4 pad
// columns on either side (row pitch 136 floats = 544 bytes, a TMA-friendly
// multiple of 16).  Warp w owns the 10-row strip w of the region and lane l
// the 4 columns 4l .. 4l+3, so a warp's row is 512 contiguous bytes: the
// south values arrive with one conflict-free 16-byte load, the new values
// leave with one 16-byte store, the west neighbour of the lane's first cell
// and the east neighbour of its last come from the adjacent lanes' registers
// (shuffles), and only lanes 0 and 31 read theirs from shared memory (one
// wavefront).  The thread keeps its 40 power values in registers and walks
// its strip with the north / centre / south values in registers.  Every
// step recomputes the whole region; cells at distance d from the region
// border are exact for d >= steps (pad and stale values only reach inward
// one cell per step), and the 112 x 64 centre is at distance >= 8.  A cell
// on the grid edge takes itself as the missing neighbour, so tiles on the
// grid edge need no halo there.
constexpr int kTileW = 112;              // output columns per tile
constexpr int kTileH = 64;               // output rows per tile
constexpr int kHalo = 8;                 // steps per launch at most
constexpr int kRegW = kTileW + 2 * kHalo;  // 128: region width (32 lanes x 4)
constexpr int kRegH = kTileH + 2 * kHalo;  // 80: region height
constexpr int kColOff = 4;               // region column 0 sits at buffer column 4
constexpr int kPitch = kRegW + 2 * kColOff;  // 136 floats per buffer row
constexpr int kBufRows = kRegH + 2;      // 82: region + pad row above and below
constexpr int kStripRows = 10;           // rows per thread
constexpr int kBlockThreads = 32 * (kRegH / kStripRows);   // 256: one warp per strip
constexpr int kBufBytes = kBufRows * kPitch * 4;            // 44,608
constexpr int kTiledSmem = 2 * kBufBytes + 64 + 128;        // two buffers, barrier, alignment
static_assert(kRegW == 32 * 4 && kRegH % kStripRows == 0, "a warp row covers the region");
static_assert((kPitch * 4) % 16 == 0 && (kColOff * 4) % 16 == 0, "16-byte rows and cells");

__device__ __forceinline__ float4 lds4(const float* p) {
  return *reinterpret_cast<const float4*>(p);
}

// Buffer (row, col) of region cell (li, lj): (li + 1, lj + kColOff).  The
// buffer covers grid rows r0 - 1 .. r0 + 80 and columns c0 - 4 .. c0 + 131,
// r0 / c0 the grid coordinates of region cell (0, 0).
template <bool kEdge>
__device__ __forceinline__ const float* advance(float* A, float* B,
                                                const float (&p)[kStripRows][4], int steps,
                                                int r0, int c0, int rows, int cols,
                                                const Coef& k) {
  const int lane = threadIdx.x & 31, strip = threadIdx.x >> 5;
  const int sc = kColOff + 4 * lane;              // buffer column of the first cell
  const int br0 = 1 + strip * kStripRows;         // first buffer row of the strip
  const int gi0 = r0 + strip * kStripRows, gj0 = c0 + 4 * lane;
  const int eoff = lane == 0 ? -1 : 4;            // lanes 0 / 31: west / east in memory
  const Coef2 k2{make_float2(k.c, k.c), make_float2(k.gx, k.gx), make_float2(k.gy, k.gy),
                 make_float2(k.gz, k.gz), make_float2(k.amb, k.amb)};
  float* cur = A;
  float* nxt = B;
  for (int s = 0; s < steps; ++s) {
    const float* col = cur + br0 * kPitch + sc;
    float4 tn = lds4(col - kPitch), tc = lds4(col);
#pragma unroll
    for (int i = 0; i < kStripRows; ++i) {
      const float4 ts = lds4(col + (i + 1) * kPitch);
      float edge = 0.f;
      if (lane == 0 || lane == 31) edge = col[i * kPitch + eoff];
      float w0 = __shfl_up_sync(0xffffffffu, tc.w, 1);
      float e3 = __shfl_down_sync(0xffffffffu, tc.x, 1);
      if (lane == 0) w0 = edge;
      if (lane == 31) e3 = edge;
      const float t[4] = {tc.x, tc.y, tc.z, tc.w};
      float n[4] = {tn.x, tn.y, tn.z, tn.w};
      float so[4] = {ts.x, ts.y, ts.z, ts.w};
      float w[4] = {w0, tc.x, tc.y, tc.z};
      float e[4] = {tc.y, tc.z, tc.w, e3};
      if (kEdge) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int gi = gi0 + i, gj = gj0 + q;
          if (gi <= 0) n[q] = t[q];
          if (gi >= rows - 1) so[q] = t[q];
          if (gj <= 0) w[q] = t[q];
          if (gj >= cols - 1) e[q] = t[q];
        }
      }
      const float2 o01 = cell_update2(make_float2(t[0], t[1]), make_float2(n[0], n[1]),
                                      make_float2(so[0], so[1]), make_float2(w[0], w[1]),
                                      make_float2(e[0], e[1]), make_float2(p[i][0], p[i][1]), k2);
      const float2 o23 = cell_update2(make_float2(t[2], t[3]), make_float2(n[2], n[3]),
                                      make_float2(so[2], so[3]), make_float2(w[2], w[3]),
                                      make_float2(e[2], e[3]), make_float2(p[i][2], p[i][3]), k2);
      *reinterpret_cast<float4*>(nxt + (br0 + i) * kPitch + sc) =
          make_float4(o01.x, o01.y, o23.x, o23.y);
      tn = tc;
      tc = ts;
    }
    __syncthreads();
    float* tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
  return cur;
}

// The thread's power values (0 outside the grid).
__device__ __forceinline__ void load_power(const float* __restrict__ P, int r0, int c0, int rows,
                                           int cols, float (&p)[kStripRows][4]) {
  const int lane = threadIdx.x & 31, strip = threadIdx.x >> 5;
  const int gj0 = c0 + 4 * lane;
#pragma unroll
  for (int i = 0; i < kStripRows; ++i) {
    const int gi = r0 + strip * kStripRows + i;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gj = gj0 + q;
      p[i][q] = (gi >= 0 && gi < rows && gj >= 0 && gj < cols)
                    ? __ldg(P + static_cast<int64_t>(gi) * cols + gj)
                    : 0.f;
    }
  }
}

// Writes the tile's 112 x 64 centre (cells inside the grid).
__device__ __forceinline__ void store_centre(const float* buf, float* out, int tr, int tc,
                                             int rows, int cols) {
  for (int idx = threadIdx.x; idx < kTileW * kTileH; idx += kBlockThreads) {
    const int li = idx / kTileW, lj = idx % kTileW;
    const int gi = tr + li, gj = tc + lj;
    if (gi < rows && gj < cols)
      out[static_cast<int64_t>(gi) * cols + gj] =
          buf[(li + kHalo + 1) * kPitch + lj + kHalo + kColOff];
  }
}

__device__ __forceinline__ bool edge_tile(int r0, int c0, int rows, int cols) {
  return r0 <= 0 || c0 <= 0 || r0 + kRegH >= rows || c0 + kRegW >= cols;
}

__global__ void __launch_bounds__(kBlockThreads, 2)
    stencil_tiled_kernel(const float* __restrict__ T, const float* __restrict__ P,
                         float* __restrict__ out, int rows, int cols, int steps, Coef k) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  float* A = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) &
                                      ~static_cast<uintptr_t>(127));
  float* B = A + kBufRows * kPitch;
  const int tr = blockIdx.y * kTileH, tc = blockIdx.x * kTileW;
  const int r0 = tr - kHalo, c0 = tc - kHalo;
  // buffer rows r0-1 .. r0+80, columns c0-4 .. c0+131 (0 outside the grid)
  for (int idx = threadIdx.x; idx < kBufRows * kPitch; idx += kBlockThreads) {
    const int bi = idx / kPitch, bj = idx % kPitch;
    const int gi = r0 - 1 + bi, gj = c0 - kColOff + bj;
    A[idx] = (gi >= 0 && gi < rows && gj >= 0 && gj < cols)
                 ? __ldg(T + static_cast<int64_t>(gi) * cols + gj)
                 : 0.f;
  }
  float p[kStripRows][4];
  load_power(P, r0, c0, rows, cols, p);
  __syncthreads();
  const float* res = edge_tile(r0, c0, rows, cols)
                         ? advance<true>(A, B, p, steps, r0, c0, rows, cols, k)
                         : advance<false>(A, B, p, steps, r0, c0, rows, cols, k);
  store_centre(res, out, tr, tc, rows, cols);
}

struct TmaMaps {
  CUtensorMap t;
};

__global__ void __launch_bounds__(kBlockThreads, 2)
    stencil_tma_kernel(const __grid_constant__ TmaMaps maps, const float* __restrict__ P,
                       float* __restrict__ out, int rows, int cols, int steps, Coef k,
                       int* err_word, unsigned long long budget_ns) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  // TMA writes to 128-byte aligned shared memory
  float* A = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) &
                                      ~static_cast<uintptr_t>(127));
  float* B = A + kBufRows * kPitch;
  uint64_t* bar = reinterpret_cast<uint64_t*>(B + kBufRows * kPitch);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bar + 1);
  const int tr = blockIdx.y * kTileH, tc = blockIdx.x * kTileW;
  const int r0 = tr - kHalo, c0 = tc - kHalo;
  if (threadIdx.x == 0) {
    dev::mbar_init(bar, 1);
    *abort_flag = 0;
    dev::fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // one 136 x 82 box at x = c0 - 4 (a multiple of 4 floats: 16 bytes),
    // y = r0 - 1; cells outside the grid read as zero
    dev::mbar_arrive_expect_tx(bar, kBufBytes);
    dev::tma_load_2d(A, &maps.t, bar, c0 - kColOff, r0 - 1);
  }
  float p[kStripRows][4];
  load_power(P, r0, c0, rows, cols, p);   // overlaps the box load
  const dev::WaitCtx w{abort_flag, err_word, budget_ns};
  const bool ok = dev::mbar_wait(bar, 0, w);
  __syncthreads();
  if (!ok) {
    // let the copy land before the CTA's shared memory goes away
    if (threadIdx.x == 0) {
      const uint64_t t0 = dev::globaltimer_ns();
      while (!dev::mbar_try_wait(bar, 0) && dev::globaltimer_ns() - t0 < budget_ns) {
      }
    }
    __syncthreads();
    return;
  }
  const float* res = edge_tile(r0, c0, rows, cols)
                         ? advance<true>(A, B, p, steps, r0, c0, rows, cols, k)
                         : advance<false>(A, B, p, steps, r0, c0, rows, cols, k);
  store_centre(res, out, tr, tc, rows, cols);
}

Coef coef_of(const compar_stencil_params_t& p) { return Coef{p.c, p.gx, p.gy, p.gz, p.amb}; }

}  // namespace

int stencil_launch(int v, int64_t rows64, int64_t cols64, int iters,
                   const compar_stencil_params_t& prm, const float* T_in, const float* P,
                   float* T_out, float* tmp, const DeviceGuard& g, cudaStream_t s) {
  const int rows = static_cast<int>(rows64), cols = static_cast<int>(cols64);
  if (rows == 0 || cols == 0) return COMPAR_OK;
  const size_t bytes = static_cast<size_t>(rows) * cols * sizeof(float);
  if (iters == 0) {
    if (T_out != T_in) COMPAR_CUDA_TRY(cudaMemcpyAsync(T_out, T_in, bytes, cudaMemcpyDeviceToDevice, s));
    return COMPAR_OK;
  }
  const Coef k = coef_of(prm);
  const int per = v == COMPAR_S_NAIVE ? 1 : kHalo;  // steps per launch
  const int launches = (iters + per - 1) / per;
  // launch l reads src and writes dst; the last launch writes T_out
  const float* src = T_in;
  cudaEvent_t ev = g.prof ? g.prof->begin(s) : nullptr;
  for (int l = 0; l < launches; ++l) {
    float* dst = ((launches - 1 - l) % 2 == 0) ? T_out : tmp;
    const int steps = std::min(per, iters - l * per);
    if (v == COMPAR_S_NAIVE) {
      const dim3 block(32, 8);
      const dim3 grid((cols + 31) / 32, (rows + 7) / 8);
      stencil_naive_kernel<<<grid, block, 0, s>>>(src, P, dst, rows, cols, k);
    } else {
      const dim3 grid((cols + kTileW - 1) / kTileW, (rows + kTileH - 1) / kTileH);
      if (v == COMPAR_S_TILED) {
        COMPAR_CUDA_TRY(smem_opt_in(reinterpret_cast<const void*>(stencil_tiled_kernel), kTiledSmem));
        stencil_tiled_kernel<<<grid, kBlockThreads, kTiledSmem, s>>>(src, P, dst, rows, cols,
                                                                       steps, k);
      } else {
        COMPAR_CUDA_TRY(smem_opt_in(reinterpret_cast<const void*>(stencil_tma_kernel), kTiledSmem));
        TmaMaps maps;
        const int rc = tma_encode_2d(&maps.t, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, src, cols, rows,
                                     cols, kPitch, kBufRows, 0);
        if (rc != COMPAR_OK) return rc;
        stencil_tma_kernel<<<grid, kBlockThreads, kTiledSmem, s>>>(
            maps, P, dst, rows, cols, steps, k, g.err_word, g.budget_ns);
      }
    }
    COMPAR_CUDA_TRY(cudaGetLastError());
    count_launch();
    src = dst;
  }
  if (g.prof) g.prof->end(ev, s, kStencilProfileBase + v);
  return COMPAR_OK;
}

bool stencil_supported(int v, int64_t rows, int64_t cols, bool aligned16) {
  if (rows > (1 << 30) || cols > (1 << 30) || rows * cols > (int64_t(1) << 34)) return false;
  switch (v) {
    case COMPAR_S_NAIVE: return (rows + 7) / 8 <= 65535;
    case COMPAR_S_TILED: return (rows + kTileH - 1) / kTileH <= 65535;
    case COMPAR_S_TMA:
      // TMA needs 16-byte aligned grids and rows (cols a multiple of 4)
      return tma_available() && aligned16 && (cols % 4 == 0) &&
             (rows + kTileH - 1) / kTileH <= 65535;
    default: return false;
  }
}

}  // namespace compar
