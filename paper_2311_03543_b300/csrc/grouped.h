// Device descriptors of the grouped (batched) GEMM path.
#pragma once

#include <cuda.h>

#include <cstdint>

#include "common.h"

namespace compar {

// Bytes of K per pipeline stage and operand row in the grouped kernel (the
// TMA / MMA swizzle width: 64 -> 64-byte swizzle, 128 -> 128-byte).
constexpr int kGroupedRow = 64;

// One problem of a grouped launch.  Tensor maps cover the K-major operands
// (A: M x K, B re-laid out as N x K); map_a2 / map_b2 are the lo pieces of
// the 3xBF16 mode.  Tiles of all problems form one list; this problem owns
// tiles [tile_start, tile_start + tiles_m * tiles_n), column-major by tile.
// (CUtensorMap members make the struct 128-byte aligned, as TMA requires.)
struct GroupProblem {
  CUtensorMap map_a, map_b, map_a2, map_b2;
  int M, N, K, num_kb;
  int tiles_m, tiles_n, tile_start, mode;  // mode: 0 bf16, 1 3xbf16, 2 tf32
  float* C;
  int64_t ldc;
  float alpha, beta;
};

// One operand re-layout of the grouped pre-pass: converts `rows x cols` of
// `src` (row pitch ld_src) into dst (and dst_lo for the split), transposing
// when asked; owns 64x64 tiles [tile_start, tile_start + tiles) of the
// batch's tile list.
struct PrepassJob {
  const void* src;
  void* dst;
  void* dst_lo;
  int64_t ld_src, ld_dst;
  int rows, cols;
  int in_type;    // COMPAR_F32 or COMPAR_BF16
  int out_kind;   // PrepassOut
  int transpose;
  int tile_start;
  int tiles_c;    // tiles along cols
  int tiles;
  int vec;        // src rows 16-byte aligned (f32) / 8-byte (bf16): 4-wide loads
};

int grouped_smem_bytes(int bn);
// d_tile_ctr: one device int, the launch's tile counter (zeroed on `s`
// before the kernel).
int launch_grouped_gemm(int bn, const GroupProblem* d_probs, int count, int total_tiles,
                        int* d_tile_ctr, const DeviceGuard& g, int num_sms, cudaStream_t s);
// transpose: some job transposes (the kernel then stages tiles in shared
// memory; without, it uses none).
int launch_grouped_prepass(const PrepassJob* d_jobs, int njobs, int total_tiles, int num_sms,
                           bool transpose, cudaStream_t s);

}  // namespace compar
