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
//   TILED : temporal blocking: a CTA loads a (64+2h) x (64+2h) region of T
//           and P into shared memory and advances it h <= 8 steps there (the
//           valid region shrinks by one cell per step), writing the 64 x 64
//           centre; ceil(steps / 8) launches.
//   TMA   : TILED with the region loaded by two TMA boxes (T and P) into
//           shared memory, completion on an mbarrier (bounded wait).
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
constexpr int kTile = 64;            // output cells per side
constexpr int kHalo = 8;             // steps per launch at most
constexpr int kReg = kTile + 2 * kHalo;  // 80: region side
constexpr int kBlockThreads = 256;
constexpr int kRegionBytes = kReg * kReg * 4;
constexpr int kTiledSmem = 3 * kRegionBytes + 64 + 128;  // T ping, T pong, P, barrier, alignment

// Advances the region in shared memory by `steps` steps.  Region cell
// (li, lj) is grid cell (r0 + li, c0 + lj) with r0 = tile row - kHalo.  At
// step s the cells at distance >= s from the region border are computed
// (their neighbours were valid after step s-1); a neighbour outside the grid
// is the cell itself, so grid-edge cells never need a halo.
__device__ __forceinline__ float* advance(float* Ta, float* Tb, const float* Ps, int steps,
                                          int r0, int c0, int rows, int cols, const Coef& k) {
  float* cur = Ta;
  float* nxt = Tb;
  for (int s = 1; s <= steps; ++s) {
    const int lo = s, hi = kReg - s;  // computed region [lo, hi) in both dims
    for (int li = lo + static_cast<int>(threadIdx.x) / 32; li < hi; li += kBlockThreads / 32) {
      const int gi = r0 + li;
      if (gi < 0 || gi >= rows) continue;
      const float* row = cur + li * kReg;
      const float* up = gi > 0 ? row - kReg : row;
      const float* dn = gi < rows - 1 ? row + kReg : row;
      for (int lj = lo + static_cast<int>(threadIdx.x % 32); lj < hi; lj += 32) {
        const int gj = c0 + lj;
        if (gj < 0 || gj >= cols) continue;
        const float t = row[lj];
        const float w = gj > 0 ? row[lj - 1] : t;
        const float e = gj < cols - 1 ? row[lj + 1] : t;
        nxt[li * kReg + lj] = cell_update(t, up[lj], dn[lj], w, e, Ps[li * kReg + lj], k);
      }
    }
    __syncthreads();
    float* tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
  return cur;
}

// Writes the tile's centre (cells inside the grid) from the region.
__device__ __forceinline__ void store_centre(const float* reg, float* out, int tr, int tc,
                                             int rows, int cols) {
  for (int li = static_cast<int>(threadIdx.x) / 32; li < kTile; li += kBlockThreads / 32) {
    const int gi = tr + li;
    if (gi >= rows) break;
    for (int lj = static_cast<int>(threadIdx.x % 32); lj < kTile; lj += 32) {
      const int gj = tc + lj;
      if (gj < cols)
        out[static_cast<int64_t>(gi) * cols + gj] = reg[(li + kHalo) * kReg + lj + kHalo];
    }
  }
}

__global__ void __launch_bounds__(kBlockThreads)
    stencil_tiled_kernel(const float* __restrict__ T, const float* __restrict__ P,
                         float* __restrict__ out, int rows, int cols, int steps, Coef k) {
  extern __shared__ __align__(128) uint8_t smem[];
  float* Ta = reinterpret_cast<float*>(smem);
  float* Tb = Ta + kReg * kReg;
  float* Ps = Tb + kReg * kReg;
  const int tr = blockIdx.y * kTile, tc = blockIdx.x * kTile;
  const int r0 = tr - kHalo, c0 = tc - kHalo;
  for (int idx = threadIdx.x; idx < kReg * kReg; idx += kBlockThreads) {
    const int li = idx / kReg, lj = idx % kReg;
    const int gi = r0 + li, gj = c0 + lj;
    float t = 0.f, p = 0.f;
    if (gi >= 0 && gi < rows && gj >= 0 && gj < cols) {
      const int64_t g = static_cast<int64_t>(gi) * cols + gj;
      t = __ldg(T + g);
      p = __ldg(P + g);
    }
    Ta[idx] = t;
    Ps[idx] = p;
  }
  __syncthreads();
  const float* res = advance(Ta, Tb, Ps, steps, r0, c0, rows, cols, k);
  store_centre(res, out, tr, tc, rows, cols);
}

struct TmaMaps {
  CUtensorMap t, p;
};

__global__ void __launch_bounds__(kBlockThreads)
    stencil_tma_kernel(const __grid_constant__ TmaMaps maps, float* __restrict__ out, int rows,
                       int cols, int steps, Coef k, int* err_word,
                       unsigned long long budget_ns) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  // TMA writes to 128-byte aligned shared memory
  float* Ta = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) &
                                       ~static_cast<uintptr_t>(127));
  float* Tb = Ta + kReg * kReg;
  float* Ps = Tb + kReg * kReg;
  uint64_t* bar = reinterpret_cast<uint64_t*>(Ps + kReg * kReg);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bar + 1);
  const int tr = blockIdx.y * kTile, tc = blockIdx.x * kTile;
  const int r0 = tr - kHalo, c0 = tc - kHalo;
  if (threadIdx.x == 0) {
    dev::mbar_init(bar, 1);
    *abort_flag = 0;
    dev::fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // x = c0 is a multiple of 8 elements (32 bytes); cells outside the grid
    // read as zero and are never used
    dev::mbar_arrive_expect_tx(bar, 2 * kRegionBytes);
    dev::tma_load_2d(Ta, &maps.t, bar, c0, r0);
    dev::tma_load_2d(Ps, &maps.p, bar, c0, r0);
  }
  const dev::WaitCtx w{abort_flag, err_word, budget_ns};
  const bool ok = dev::mbar_wait(bar, 0, w);
  __syncthreads();
  if (!ok) {
    // let the copies land before the CTA's shared memory goes away
    if (threadIdx.x == 0) {
      const uint64_t t0 = dev::globaltimer_ns();
      while (!dev::mbar_try_wait(bar, 0) && dev::globaltimer_ns() - t0 < budget_ns) {
      }
    }
    __syncthreads();
    return;
  }
  const float* res = advance(Ta, Tb, Ps, steps, r0, c0, rows, cols, k);
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
      const dim3 grid((cols + kTile - 1) / kTile, (rows + kTile - 1) / kTile);
      if (v == COMPAR_S_TILED) {
        static bool attr = false;
        if (!attr) {
          COMPAR_CUDA_TRY(cudaFuncSetAttribute(stencil_tiled_kernel,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               kTiledSmem));
          attr = true;
        }
        stencil_tiled_kernel<<<grid, kBlockThreads, kTiledSmem, s>>>(src, P, dst, rows, cols,
                                                                       steps, k);
      } else {
        static bool attr = false;
        if (!attr) {
          COMPAR_CUDA_TRY(cudaFuncSetAttribute(stencil_tma_kernel,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               kTiledSmem));
          attr = true;
        }
        TmaMaps maps;
        int rc = tma_encode_2d(&maps.t, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, src, cols, rows, cols,
                               kReg, kReg, 0);
        if (rc == COMPAR_OK)
          rc = tma_encode_2d(&maps.p, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, P, cols, rows, cols,
                             kReg, kReg, 0);
        if (rc != COMPAR_OK) return rc;
        stencil_tma_kernel<<<grid, kBlockThreads, kTiledSmem, s>>>(maps, dst, rows, cols, steps,
                                                                     k, g.err_word, g.budget_ns);
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
    case COMPAR_S_TILED: return (rows + kTile - 1) / kTile <= 65535;
    case COMPAR_S_TMA:
      // TMA needs 16-byte aligned grids and rows (cols a multiple of 4)
      return tma_available() && aligned16 && (cols % 4 == 0) &&
             (rows + kTile - 1) / kTile <= 65535;
    default: return false;
  }
}

}  // namespace compar
