// FP32 SIMT implementation variants of C = alpha*A*B + beta*C (the
// matrix-multiply component of Sec. 2.1 / Table 2; the paper's own GPU
// variant of it is a hand-written CUDA kernel for a Pascal GPU).
//
//  * gemm_naive_kernel: one thread per C element, FP32 FMA over k.
//  * gemm_simt_kernel : shared-memory tiled, register-blocked, with 128-bit
//    global loads and double-buffered shared-memory tiles; optional split-K
//    with a separate reduction pass.
//  * gemm_skinny_kernel: the same variant's plan for a few rows of A against
//    a wide, deep B, built to stream B from HBM once (split K, cluster sums
//    through distributed shared memory).
//
// Row-major A (M x K, lda), B (K x N, ldb), C (M x N, ldc).  Inputs may be
// float32, bf16 (uint16 bit patterns) or E4M3 (bytes); they are widened to
// float32 on load and every product and sum is an FP32 FMA.
#include <cooperative_groups.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "common.h"
#include "ptx.cuh"

namespace compar {
namespace {

// ------------------------------------------------------------------ element types
__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(uint16_t b) {  // bf16: the high half of a float32
  return __uint_as_float(static_cast<uint32_t>(b) << 16);
}
__device__ __forceinline__ float to_f32(uint8_t c) {   // E4M3 -> half (exact) -> float
  const __half_raw h = __nv_cvt_fp8_to_halfraw(static_cast<__nv_fp8_storage_t>(c), __NV_E4M3);
  return __half2float(__half(h));
}
template <typename T>
__device__ __forceinline__ float ld1(const T* p) { return to_f32(__ldg(p)); }

// Four consecutive elements with one aligned load (16, 8 or 4 bytes).
__device__ __forceinline__ void ld4(const float* p, float (&o)[4]) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4(const uint16_t* p, float (&o)[4]) {
  const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
  o[0] = __uint_as_float(v.x << 16); o[1] = __uint_as_float(v.x & 0xFFFF0000u);
  o[2] = __uint_as_float(v.y << 16); o[3] = __uint_as_float(v.y & 0xFFFF0000u);
}
__device__ __forceinline__ void ld4(const uint8_t* p, float (&o)[4]) {
  const uint32_t v = __ldg(reinterpret_cast<const unsigned int*>(p));
#pragma unroll
  for (int q = 0; q < 4; ++q) o[q] = to_f32(static_cast<uint8_t>(v >> (8 * q)));
}

// ------------------------------------------------------------------ naive
template <typename T>
__global__ void gemm_naive_kernel(int M, int N, int K, float alpha, const T* __restrict__ A,
                                  int64_t lda, const T* __restrict__ B, int64_t ldb,
                                  float beta, float* __restrict__ C, int64_t ldc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= M || j >= N) return;
  const T* a = A + static_cast<int64_t>(i) * lda;
  float acc = 0.f;
  for (int p = 0; p < K; ++p) acc = fmaf(ld1(a + p), ld1(B + static_cast<int64_t>(p) * ldb + j), acc);
  float* c = C + static_cast<int64_t>(i) * ldc + j;
  *c = (beta == 0.f) ? alpha * acc : fmaf(alpha, acc, beta * *c);
}

__global__ void scale_c_kernel(float* C, int M, int N, int64_t ldc, float beta) {
  const int64_t total = static_cast<int64_t>(M) * N;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = t / N, j = t % N;
    float* c = C + i * ldc + j;
    *c = (beta == 0.f) ? 0.f : beta * *c;
  }
}

// ------------------------------------------------------------------ tiled
// Thread (ty, tx) owns TM x TN outputs laid out as groups of 4 rows strided
// by 4*(BM/TM) and groups of 4 columns strided by 4*(BN/TN), so that its
// shared-memory reads are 128-bit and a warp's B reads cover distinct banks.
template <int BM, int BN, int BK, int TM, int TN, bool VEC>
struct SimtCfg {
  static constexpr int kThreadsX = BN / TN;
  static constexpr int kThreadsY = BM / TM;
  static constexpr int kThreads = kThreadsX * kThreadsY;
  static constexpr int kRowStride = 4 * kThreadsY;  // between 4-row groups
  static constexpr int kColStride = 4 * kThreadsX;
  static constexpr int kAElems = BM * BK / kThreads;  // A elements loaded per thread
  static constexpr int kBElems = BK * BN / kThreads;
  static_assert(TM % 4 == 0 && TN % 4 == 0, "micro tile in 4-wide groups");
  static_assert(kAElems % 4 == 0 && kBElems % 4 == 0, "vector loads");
  static_assert(BM % 32 == 0, "row swizzle of the A tile");
};

// The A tile is stored transposed (As[k][m]); row m of K column k sits at
// m ^ a_swizzle<BK>(k).  Each thread stores 4 K columns of one row, so a
// warp's 32 stores of one K offset cover 32 * 4 / BK rows and BK / 4 column
// groups; without the swizzle they hit only 32 * 4 / BK banks.  XOR-ing the
// row with (k / 4) x (128 / BK) spreads them over all 32; multiples of 4
// keep the 4-row groups that the FMA loop reads as float4 contiguous.
template <int BK>
__device__ __forceinline__ int a_swizzle(int k) {
  static_assert(BK == 16 || BK == 32, "K tile of 16 or 32");
  return ((k >> 2) & (BK / 4 - 1)) * (128 / BK);
}

template <typename T, int BM, int BN, int BK, int TM, int TN, bool VEC>
// One CTA per SM, so the 8 x 8 micro-tile, its fragments and the next
// tile's prefetch registers fit without spills (capped at 128 registers for
// two CTAs per SM the kernel spilled and ran 7 % slower on 4096^3).
__global__ void __launch_bounds__(SimtCfg<BM, BN, BK, TM, TN, VEC>::kThreads, 1)
    gemm_simt_kernel(int M, int N, int K, int k_per_split, float alpha,
                     const T* __restrict__ A, int64_t lda, const T* __restrict__ B,
                     int64_t ldb, float beta, float* __restrict__ C, int64_t ldc,
                     float* __restrict__ partial) {
  using Cfg = SimtCfg<BM, BN, BK, TM, TN, VEC>;
  __shared__ __align__(16) float As[2][BK][BM];
  __shared__ __align__(16) float Bs[2][BK][BN];

  const int tid = threadIdx.x;
  const int tx = tid % Cfg::kThreadsX;
  const int ty = tid / Cfg::kThreadsX;
  const int m0 = blockIdx.y * BM;
  const int n0 = blockIdx.x * BN;
  const int k_begin = blockIdx.z * k_per_split;
  const int k_end = min(K, k_begin + k_per_split);

  float ra[Cfg::kAElems];
  float rb[Cfg::kBElems];

  // A tile: BM rows x BK columns; linear element e -> (row e / BK, col e % BK)
  auto load_a = [&](int k0) {
#pragma unroll
    for (int v = 0; v < Cfg::kAElems / 4; ++v) {
      const int e = (v * Cfg::kThreads + tid) * 4;
      const int r = e / BK, c = e % BK;
      const int gi = m0 + r, gk = k0 + c;
      if constexpr (VEC) {
        float x[4] = {0.f, 0.f, 0.f, 0.f};
        if (gi < M && gk < k_end) ld4(A + static_cast<int64_t>(gi) * lda + gk, x);
        ra[4 * v + 0] = x[0]; ra[4 * v + 1] = x[1]; ra[4 * v + 2] = x[2]; ra[4 * v + 3] = x[3];
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          ra[4 * v + q] = (gi < M && gk + q < k_end)
                              ? ld1(A + static_cast<int64_t>(gi) * lda + gk + q) : 0.f;
      }
    }
  };
  auto store_a = [&](int buf) {
#pragma unroll
    for (int v = 0; v < Cfg::kAElems / 4; ++v) {
      const int e = (v * Cfg::kThreads + tid) * 4;
      const int r = e / BK, c = e % BK;
#pragma unroll
      for (int q = 0; q < 4; ++q) As[buf][c + q][r ^ a_swizzle<BK>(c + q)] = ra[4 * v + q];
    }
  };
  // B tile: BK rows x BN columns
  auto load_b = [&](int k0) {
#pragma unroll
    for (int v = 0; v < Cfg::kBElems / 4; ++v) {
      const int e = (v * Cfg::kThreads + tid) * 4;
      const int r = e / BN, c = e % BN;
      const int gk = k0 + r, gj = n0 + c;
      if constexpr (VEC) {
        float x[4] = {0.f, 0.f, 0.f, 0.f};
        if (gk < k_end && gj < N) ld4(B + static_cast<int64_t>(gk) * ldb + gj, x);
        rb[4 * v + 0] = x[0]; rb[4 * v + 1] = x[1]; rb[4 * v + 2] = x[2]; rb[4 * v + 3] = x[3];
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          rb[4 * v + q] = (gk < k_end && gj + q < N)
                              ? ld1(B + static_cast<int64_t>(gk) * ldb + gj + q) : 0.f;
      }
    }
  };
  auto store_b = [&](int buf) {
#pragma unroll
    for (int v = 0; v < Cfg::kBElems / 4; ++v) {
      const int e = (v * Cfg::kThreads + tid) * 4;
      const int r = e / BN, c = e % BN;
      *reinterpret_cast<float4*>(&Bs[buf][r][c]) =
          make_float4(rb[4 * v + 0], rb[4 * v + 1], rb[4 * v + 2], rb[4 * v + 3]);
    }
  };

  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

  int buf = 0;
  if (k_begin < k_end) {
    load_a(k_begin);
    load_b(k_begin);
    store_a(0);
    store_b(0);
  }
  __syncthreads();

  for (int k0 = k_begin; k0 < k_end; k0 += BK) {
    const bool has_next = k0 + BK < k_end;
    if (has_next) {
      load_a(k0 + BK);
      load_b(k0 + BK);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[TM], b[TN];
#pragma unroll
      for (int g = 0; g < TM / 4; ++g) {
        const float4 x = *reinterpret_cast<const float4*>(
            &As[buf][kk][(ty * 4 + g * Cfg::kRowStride) ^ a_swizzle<BK>(kk)]);
        a[4 * g + 0] = x.x; a[4 * g + 1] = x.y; a[4 * g + 2] = x.z; a[4 * g + 3] = x.w;
      }
#pragma unroll
      for (int g = 0; g < TN / 4; ++g) {
        const float4 x = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4 + g * Cfg::kColStride]);
        b[4 * g + 0] = x.x; b[4 * g + 1] = x.y; b[4 * g + 2] = x.z; b[4 * g + 3] = x.w;
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (has_next) {
      store_a(buf ^ 1);
      store_b(buf ^ 1);
    }
    __syncthreads();
    buf ^= 1;
  }

  // Epilogue: each thread writes its 4-wide column groups; split-K writes raw
  // partial sums to its slice of the workspace instead of C.
  const bool vec_store = VEC && partial == nullptr;
#pragma unroll
  for (int gi = 0; gi < TM / 4; ++gi) {
#pragma unroll
    for (int ii = 0; ii < 4; ++ii) {
      const int row = m0 + ty * 4 + gi * Cfg::kRowStride + ii;
      if (row >= M) continue;
#pragma unroll
      for (int gj = 0; gj < TN / 4; ++gj) {
        const int col = n0 + tx * 4 + gj * Cfg::kColStride;
        const float* v = &acc[gi * 4 + ii][gj * 4];
        if (partial != nullptr) {
          float* p = partial + (static_cast<int64_t>(blockIdx.z) * M + row) * N + col;
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (col + q < N) p[q] = v[q];
        } else if (vec_store && col + 3 < N) {
          float4* c4 = reinterpret_cast<float4*>(C + static_cast<int64_t>(row) * ldc + col);
          float4 out;
          if (beta == 0.f) {
            out = make_float4(alpha * v[0], alpha * v[1], alpha * v[2], alpha * v[3]);
          } else {
            const float4 old = *c4;
            out = make_float4(fmaf(alpha, v[0], beta * old.x), fmaf(alpha, v[1], beta * old.y),
                              fmaf(alpha, v[2], beta * old.z), fmaf(alpha, v[3], beta * old.w));
          }
          *c4 = out;
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (col + q >= N) break;
            float* c = C + static_cast<int64_t>(row) * ldc + col + q;
            *c = (beta == 0.f) ? alpha * v[q] : fmaf(alpha, v[q], beta * *c);
          }
        }
      }
    }
  }
}


// ------------------------------------------------------------------ skinny M
// A few rows of A against a wide, deep B: the work is bound by reading B once
// from HBM (4 K N bytes for float32 against 2 M N K flop; at M = 16 the FMA
// pipe needs about 0.7 of the time the copy takes).  Thread t of a CTA owns 4
// adjacent columns and MT rows of C and walks one K chunk: one vector load of
// 4 B elements per k, SkinnyUnroll<MT> loads per batch, the next batch issued
// before the current one is used.  The chunk of A sits in shared memory as
// [k][row], read with broadcast float4 loads.  Row groups are the fastest
// grid index, so the CTAs that read one B chunk for different rows run
// together and share it through L2.
//
// K is split into chunks.  The CTAs of a cluster (consecutive chunks of one
// column block) add their partial tiles through distributed shared memory in
// rank order; the cluster sums go to C when one cluster covers K, else to
// workspace slabs that splitk_reduce_kernel adds in cluster order.  Every sum
// is taken in a fixed order, so results are reproducible.
constexpr int kSkinnyThreads = 128;
constexpr int kSkinnyCols = 4 * kSkinnyThreads;  // columns of C per CTA
constexpr int kSkinnyMaxRows = 16;               // rows of C per thread (MT is 8 or 16)
constexpr int kSkinnyMaxChunk = 512;             // k per CTA (A chunk of 32 KB)
constexpr int kSkinnyMaxCluster = 8;             // portable cluster size
constexpr int kSkinnyMaxM = 64;                  // rows the plan takes this kernel for
constexpr int kSkinnyCtasPerSm = 3;
constexpr int kSkinnyLastSum = 8;  // at most this many cluster sums: added in the kernel
static_assert(kSkinnyMaxChunk >= kSkinnyCols, "the partial tile reuses the A chunk's memory");
template <int MT>
constexpr int SkinnyUnroll = MT == 8 ? 12 : 8;  // B loads per batch (registers allow)

template <int MT>
__device__ __forceinline__ void skinny_fma(float (&acc)[MT][4], const float* a_k,
                                           const float (&b)[4]) {
#pragma unroll
  for (int r = 0; r < MT; r += 4) {
    const float4 a = *reinterpret_cast<const float4*>(a_k + r);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      acc[r + 0][q] = fmaf(a.x, b[q], acc[r + 0][q]);
      acc[r + 1][q] = fmaf(a.y, b[q], acc[r + 1][q]);
      acc[r + 2][q] = fmaf(a.z, b[q], acc[r + 2][q]);
      acc[r + 3][q] = fmaf(a.w, b[q], acc[r + 3][q]);
    }
  }
}

template <typename T, int U>
__device__ __forceinline__ void skinny_load(const T* b, int64_t ldb, float (&v)[U][4]) {
#pragma unroll
  for (int u = 0; u < U; ++u) ld4(b + u * ldb, v[u]);
}

template <int MT, int U>
__device__ __forceinline__ void skinny_fma_batch(float (&acc)[MT][4], const float* a,
                                                 const float (&v)[U][4]) {
#pragma unroll
  for (int u = 0; u < U; ++u) skinny_fma<MT>(acc, a + u * MT, v[u]);
}

// Four sums of one row (columns n .. n+3) to a partial slab, or to C as
// alpha * s + beta * C.
__device__ __forceinline__ void skinny_store(const float4 s, int row, int n, int N, float alpha,
                                             float beta, float* C, int64_t ldc, bool c_vec,
                                             float* slab) {
  if (slab != nullptr) {
    *reinterpret_cast<float4*>(slab + static_cast<int64_t>(row) * N + n) = s;
    return;
  }
  float* c = C + static_cast<int64_t>(row) * ldc + n;
  const float v[4] = {s.x, s.y, s.z, s.w};
  if (c_vec) {
    float4 out;
    if (beta == 0.f) {
      out = make_float4(alpha * v[0], alpha * v[1], alpha * v[2], alpha * v[3]);
    } else {
      const float4 old = *reinterpret_cast<const float4*>(c);
      out = make_float4(fmaf(alpha, v[0], beta * old.x), fmaf(alpha, v[1], beta * old.y),
                        fmaf(alpha, v[2], beta * old.z), fmaf(alpha, v[3], beta * old.w));
    }
    *reinterpret_cast<float4*>(c) = out;
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) c[q] = (beta == 0.f) ? alpha * v[q] : fmaf(alpha, v[q], beta * c[q]);
  }
}

// Grid (row groups of MT, column blocks, K chunks); launched with clusters of
// `cluster` CTAs along K (1, 2, 4 or 8).  Needs N % 4 == 0 and B rows whose
// 4-element groups are aligned to their size (one vector load per 4 columns).
template <typename T, int MT>
__global__ void __launch_bounds__(kSkinnyThreads, kSkinnyCtasPerSm)
    gemm_skinny_kernel(int M, int N, int K, int k_chunk, int cluster, float alpha,
                       const T* __restrict__ A, int64_t lda, const T* __restrict__ B,
                       int64_t ldb, float beta, float* __restrict__ C, int64_t ldc, bool c_vec,
                       float* __restrict__ partial, unsigned long long* __restrict__ counters,
                       unsigned int epoch) {
  static_assert(MT % kSkinnyMaxCluster == 0 && MT <= kSkinnyMaxRows, "rows per thread");
  constexpr int U = SkinnyUnroll<MT>;
  __shared__ __align__(16) float sm[kSkinnyMaxChunk * MT];
  const int tid = threadIdx.x;
  const int r0 = blockIdx.x * MT;
  const int n = blockIdx.y * kSkinnyCols + 4 * tid;
  const int k0 = blockIdx.z * k_chunk;
  const int kc = max(0, min(K - k0, k_chunk));  // trailing chunks may be empty
  const bool active = n < N;
  const T* b = B + static_cast<int64_t>(k0) * ldb + n;
  const int full = kc / U * U;
  float cur[U][4], nxt[U][4];
  if (active && full > 0) skinny_load(b, ldb, cur);  // in flight while A is staged

  // the chunk of A, widened to float32, as [k][row]; rows past M read as zero
  for (int e = tid; e < kc * MT; e += kSkinnyThreads) {
    const int r = e / kc, kk = e - r * kc;
    sm[kk * MT + r] = (r0 + r < M) ? ld1(A + static_cast<int64_t>(r0 + r) * lda + k0 + kk) : 0.f;
  }
  __syncthreads();

  float acc[MT][4];
#pragma unroll
  for (int r = 0; r < MT; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[r][q] = 0.f;
  if (active) {
    for (int kk = 0; kk < full; kk += 2 * U) {
      const int k1 = kk + U;
      if (k1 < full) skinny_load(b + k1 * ldb, ldb, nxt);
      skinny_fma_batch<MT, U>(acc, sm + kk * MT, cur);
      if (k1 >= full) break;
      if (k1 + U < full) skinny_load(b + (k1 + U) * ldb, ldb, cur);
      skinny_fma_batch<MT, U>(acc, sm + k1 * MT, nxt);
    }
    for (int kk = full; kk < kc; ++kk) {
      float v[4];
      ld4(b + kk * ldb, v);
      skinny_fma<MT>(acc, sm + kk * MT, v);
    }
  }

  float* slab =
      partial ? partial + static_cast<int64_t>(blockIdx.z / cluster) * M * N : nullptr;
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  int rank = 0, row0 = 0, rows = MT;  // the rows of C this CTA writes
  if (cluster == 1) {  // the same for every CTA of the grid
    if (active)
#pragma unroll
      for (int r = 0; r < MT; ++r)
        if (r0 + r < M)
          skinny_store(make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]), r0 + r, n, N,
                       alpha, beta, C, ldc, c_vec, slab);
  } else {
    // Cluster sum: every CTA leaves its tile in shared memory as [row][column];
    // rank q adds rows [q * rows, (q + 1) * rows) over the cluster's tiles.
    __syncthreads();  // the A chunk is no longer read
#pragma unroll
    for (int r = 0; r < MT; ++r)
      *reinterpret_cast<float4*>(sm + r * kSkinnyCols + 4 * tid) =
          make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
    cl.sync();
    rows = MT / cluster;
    rank = static_cast<int>(cl.block_rank());
    row0 = rank * rows;
    for (int i = 0; i < rows; ++i) {
      const int r = row0 + i;
      float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int q = 0; q < cluster; ++q) {
        const float4 v =
            *cl.map_shared_rank(reinterpret_cast<float4*>(sm + r * kSkinnyCols) + tid, q);
        s.x += v.x;
        s.y += v.y;
        s.z += v.z;
        s.w += v.w;
      }
      if (active && r0 + r < M) skinny_store(s, r0 + r, n, N, alpha, beta, C, ldc, c_vec, slab);
    }
  }

  // With `counters`, the last cluster of this row group and column block to
  // finish adds every cluster's slab in cluster order and writes C (the same
  // sums as splitk_reduce_kernel).  No CTA waits for another: each one counts
  // its cluster's arrival and leaves unless it was the last.  A counter word
  // is (epoch << 32 | count); a word carrying another launch's epoch counts
  // as zero, so no reset is needed between calls.
  if (counters != nullptr) {
    __shared__ int last_flag;
    const unsigned int groups = gridDim.z / cluster;
    __threadfence();  // this thread's slab stores, before the arrival is counted
    if (cluster == 1) __syncthreads(); else cl.sync();
    if (rank == 0 && tid == 0) {
      unsigned long long* cnt = counters + blockIdx.y * gridDim.x + blockIdx.x;
      unsigned long long seen = *reinterpret_cast<volatile unsigned long long*>(cnt);
      unsigned int before;
      for (;;) {  // at most `groups` clusters contend for one word
        before = static_cast<unsigned int>(seen >> 32) == epoch
                     ? static_cast<unsigned int>(seen) : 0u;
        const unsigned long long next =
            (static_cast<unsigned long long>(epoch) << 32) | (before + 1u);
        const unsigned long long got = atomicCAS(cnt, seen, next);
        if (got == seen) break;
        seen = got;
      }
      last_flag = before == groups - 1;
    }
    if (cluster == 1) __syncthreads(); else cl.sync();
    const int last = cluster == 1 ? last_flag : *cl.map_shared_rank(&last_flag, 0);
    if (last) {
      __threadfence();
      for (int i = 0; i < rows; ++i) {
        const int row = r0 + row0 + i;
        if (!active || row >= M) continue;
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int g = 0; g < groups; ++g) {
          const float4 v = __ldcg(reinterpret_cast<const float4*>(
              partial + (static_cast<int64_t>(g) * M + row) * N + n));
          s.x += v.x;
          s.y += v.y;
          s.z += v.z;
          s.w += v.w;
        }
        skinny_store(s, row, n, N, alpha, beta, C, ldc, c_vec, nullptr);
      }
    }
  }
  if (cluster > 1) cl.sync();  // no CTA leaves while a peer still reads its shared memory
}

// C = alpha * sum_s partial[s] + beta * C, the slabs added in order; the
// loads of up to 8 slabs are issued together so that their latencies overlap.
// May be launched programmatically after the kernel that writes the slabs.
__global__ void splitk_reduce_kernel(int M, int N, int splits, const float* __restrict__ partial,
                                     float alpha, float beta, float* __restrict__ C, int64_t ldc) {
  dev::griddep_wait();
  dev::griddep_launch_dependents();
  constexpr int kBatch = 8;
  const int64_t total = static_cast<int64_t>(M) * N;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float s = 0.f;
    for (int z0 = 0; z0 < splits; z0 += kBatch) {
      float v[kBatch];
#pragma unroll
      for (int i = 0; i < kBatch; ++i)
        v[i] = z0 + i < splits ? __ldg(partial + (z0 + i) * total + t) : 0.f;
#pragma unroll
      for (int i = 0; i < kBatch; ++i)
        if (z0 + i < splits) s += v[i];
    }
    const int64_t i = t / N, j = t % N;
    float* c = C + i * ldc + j;
    *c = (beta == 0.f) ? alpha * s : fmaf(alpha, s, beta * *c);
  }
}

// alpha with the fp8 dequantisation factors folded in
float effective_alpha(const GemmCall& c) {
  return c.dtype == COMPAR_F8E4M3 ? c.alpha * c.scale_a * c.scale_b : c.alpha;
}

template <typename T, int BM, int BN, int BK, int TM, int TN>
int run_simt(const GemmCall& c, const SimtPlan& plan, Workspace& ws, const DeviceGuard& g,
             int num_sms, cudaStream_t s) {
  const int M = static_cast<int>(c.m), N = static_cast<int>(c.n), K = static_cast<int>(c.k);
  const int tiles_m = (M + BM - 1) / BM, tiles_n = (N + BN - 1) / BN;
  const int splits = plan.splits, k_per = static_cast<int>(plan.k_per);
  float* partial = nullptr;
  if (splits > 1) {
    const size_t need = static_cast<size_t>(splits) * M * N * sizeof(float);
    int rc = ws.ensure(need, s);
    if (rc != COMPAR_OK) return rc;
    partial = static_cast<float*>(ws.ptr);
  }
  constexpr uintptr_t kVecBytes = 4 * sizeof(T);
  const bool vec = (c.k % 4 == 0) && (c.n % 4 == 0) && (c.lda % 4 == 0) && (c.ldb % 4 == 0) &&
                   (c.ldc % 4 == 0) && (reinterpret_cast<uintptr_t>(c.A) % kVecBytes == 0) &&
                   (reinterpret_cast<uintptr_t>(c.B) % kVecBytes == 0) &&
                   (reinterpret_cast<uintptr_t>(c.C) % 16 == 0);
  dim3 grid(tiles_n, tiles_m, splits);
  constexpr int threads = SimtCfg<BM, BN, BK, TM, TN, true>::kThreads;
  const T* A = static_cast<const T*>(c.A);
  const T* B = static_cast<const T*>(c.B);
  const float alpha = effective_alpha(c);
  cudaEvent_t ev = g.prof ? g.prof->begin(s) : nullptr;
  if (vec)
    gemm_simt_kernel<T, BM, BN, BK, TM, TN, true><<<grid, threads, 0, s>>>(
        M, N, K, k_per, alpha, A, c.lda, B, c.ldb, c.beta, c.C, c.ldc, partial);
  else
    gemm_simt_kernel<T, BM, BN, BK, TM, TN, false><<<grid, threads, 0, s>>>(
        M, N, K, k_per, alpha, A, c.lda, B, c.ldb, c.beta, c.C, c.ldc, partial);
  COMPAR_CUDA_TRY(cudaGetLastError());
  if (g.prof) g.prof->end(ev, s, COMPAR_V_SIMT);
  count_launch();
  if (splits > 1) {
    const int64_t total = static_cast<int64_t>(M) * N;
    const int blocks = static_cast<int>(std::min<int64_t>((total + 255) / 256, 4 * num_sms));
    splitk_reduce_kernel<<<blocks, 256, 0, s>>>(M, N, splits, partial, alpha, c.beta, c.C,
                                                c.ldc);
    COMPAR_CUDA_TRY(cudaGetLastError());
    count_launch();
  }
  return COMPAR_OK;
}

template <typename T>
int run_naive(const GemmCall& c, const DeviceGuard& g, cudaStream_t s) {
  dim3 block(16, 16);
  cudaEvent_t ev = g.prof ? g.prof->begin(s) : nullptr;
  dim3 grid(static_cast<unsigned>((c.n + 15) / 16), static_cast<unsigned>((c.m + 15) / 16));
  gemm_naive_kernel<T><<<grid, block, 0, s>>>(
      static_cast<int>(c.m), static_cast<int>(c.n), static_cast<int>(c.k), effective_alpha(c),
      static_cast<const T*>(c.A), c.lda, static_cast<const T*>(c.B), c.ldb, c.beta, c.C, c.ldc);
  COMPAR_CUDA_TRY(cudaGetLastError());
  if (g.prof) g.prof->end(ev, s, COMPAR_V_NAIVE);
  count_launch();
  return COMPAR_OK;
}

// The skinny plan's kernel; when more than one cluster covers K, `partial`
// holds plan.splits slabs of M x N, added by the last cluster to finish when
// `counters` (one per row group and column block, with this launch's epoch) is given, else by
// the reduce pass.
template <typename T>
int run_skinny(const GemmCall& c, const SimtPlan& plan, float* partial,
               unsigned long long* counters, unsigned int epoch, int num_sms, cudaStream_t s) {
  const int M = static_cast<int>(c.m), N = static_cast<int>(c.n), K = static_cast<int>(c.k);
  const float alpha = effective_alpha(c);
  const bool c_vec = c.ldc % 4 == 0 && reinterpret_cast<uintptr_t>(c.C) % 16 == 0;
  float* slabs = plan.splits > 1 ? partial : nullptr;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((M + plan.bm - 1) / plan.bm, (N + kSkinnyCols - 1) / kSkinnyCols,
                     plan.splits * plan.cluster);
  cfg.blockDim = dim3(kSkinnyThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = plan.cluster;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  auto kernel = plan.bm == 8 ? gemm_skinny_kernel<T, 8> : gemm_skinny_kernel<T, 16>;
  COMPAR_CUDA_TRY(cudaLaunchKernelEx(&cfg, kernel, M, N, K,
                                     static_cast<int>(plan.k_per), plan.cluster, alpha,
                                     static_cast<const T*>(c.A), c.lda,
                                     static_cast<const T*>(c.B), c.ldb, c.beta, c.C, c.ldc,
                                     c_vec, slabs, plan.splits > 1 ? counters : nullptr, epoch));
  count_launch();
  if (plan.splits > 1 && counters == nullptr)
    return launch_splitk_reduce(M, N, plan.splits, partial, alpha, c.beta, c.C, c.ldc, num_sms, s);
  return COMPAR_OK;
}

template <typename T>
int dispatch_simt(const GemmCall& c, Workspace& ws, const DeviceGuard& g, int num_sms,
                  cudaStream_t s) {
  const SimtPlan plan = simt_plan(c, num_sms);
  if (plan.skinny) {
    float* partial = nullptr;
    unsigned long long* counters = nullptr;
    unsigned int epoch = 0;
    if (plan.splits > 1) {
      int rc = ws.ensure(static_cast<size_t>(plan.splits) * c.m * c.n * sizeof(float), s);
      if (rc != COMPAR_OK) return rc;
      partial = static_cast<float*>(ws.ptr);
      if (plan.splits <= kSkinnyLastSum) {  // few slabs: the last cluster adds them
        rc = ws.take_counters(static_cast<size_t>((c.m + plan.bm - 1) / plan.bm) *
                                  ((c.n + kSkinnyCols - 1) / kSkinnyCols),
                              s, &epoch);
        if (rc != COMPAR_OK) return rc;
        counters = ws.counters;
      }
    }
    cudaEvent_t ev = g.prof ? g.prof->begin(s) : nullptr;
    const int rc = run_skinny<T>(c, plan, partial, counters, epoch, num_sms, s);
    if (rc == COMPAR_OK && g.prof) g.prof->end(ev, s, COMPAR_V_SIMT);
    return rc;
  }
  if (plan.bm == 32) return run_simt<T, 32, 128, 32, 4, 8>(c, plan, ws, g, num_sms, s);
  return run_simt<T, 128, 128, 16, 8, 8>(c, plan, ws, g, num_sms, s);
}

size_t dtype_bytes(compar_dtype_t d) { return d == COMPAR_F32 ? 4 : (d == COMPAR_BF16 ? 2 : 1); }

}  // namespace

SimtPlan simt_plan(const GemmCall& c, int num_sms) {
  const int64_t m = c.m, n = c.n, k = c.k;
  SimtPlan p;
  // A few rows against a wide, deep B whose rows allow 4-element vector
  // loads: the skinny kernel, K split to fill every SM (three CTAs each),
  // chunks summed on chip in clusters of up to 8.
  const bool b_vec = n % 4 == 0 && c.ldb % 4 == 0 &&
                     reinterpret_cast<uintptr_t>(c.B) % (4 * dtype_bytes(c.dtype)) == 0;
  if (m <= kSkinnyMaxM && n >= kSkinnyCols / 2 && n <= 65535LL * kSkinnyCols && b_vec &&
      k <= static_cast<int64_t>(kSkinnyMaxChunk) * 32768) {
    p.skinny = true;
    p.bm = m <= 8 ? 8 : 16;  // rows of C per thread
    p.bn = kSkinnyCols;
    p.bk = 0;
    const int64_t ctas = ((m + p.bm - 1) / p.bm) * ((n + kSkinnyCols - 1) / kSkinnyCols);
    int64_t chunks = std::max<int64_t>(1, kSkinnyCtasPerSm * static_cast<int64_t>(num_sms) / ctas);
    chunks = std::max<int64_t>(1, std::min<int64_t>(chunks, k / 32));
    int cl = 1;
    while (cl < kSkinnyMaxCluster && 2 * cl <= chunks) cl *= 2;
    chunks = chunks / cl * cl;
    int64_t chunk = (k + chunks - 1) / chunks;
    chunk = (chunk + 7) / 8 * 8;
    chunk = std::min<int64_t>(std::max<int64_t>(chunk, 8), kSkinnyMaxChunk);
    chunks = (k + chunk - 1) / chunk;
    // a capped chunk can leave a count that is not a multiple of the
    // cluster; pad with empty chunks only while the grid still fits
    const int64_t slots = kSkinnyCtasPerSm * static_cast<int64_t>(num_sms);
    while (cl > 1 && chunks % cl != 0 && (chunks + cl - 1) / cl * cl * ctas > slots) cl /= 2;
    chunks = (chunks + cl - 1) / cl * cl;
    p.cluster = cl;
    p.splits = static_cast<int>(chunks / cl);
    p.k_per = chunk;
    return p;
  }
  // Short-M shapes take a 32-row tile so fewer rows of work are wasted.
  if (m <= 48) {
    p.bm = 32;
    p.bk = 32;
  } else {
    p.bm = 128;
    p.bk = 16;
  }
  p.bn = 128;
  p.splits = 1;
  p.k_per = k;
  // Split K when the tiles alone cannot fill the GPU and K is long.
  const int64_t tiles = ((m + p.bm - 1) / p.bm) * ((n + p.bn - 1) / p.bn);
  if (tiles < num_sms && k >= 1024) {
    int64_t sp = std::min<int64_t>((2 * static_cast<int64_t>(num_sms) + tiles - 1) / tiles, k / 256);
    sp = std::max<int64_t>(1, std::min<int64_t>(sp, 32));
    if (sp > 1) {
      p.k_per = ((k + sp - 1) / sp + p.bk - 1) / p.bk * p.bk;
      p.splits = static_cast<int>((k + p.k_per - 1) / p.k_per);
    }
  }
  return p;
}

int launch_naive(const GemmCall& c, const DeviceGuard& g, cudaStream_t s) {
  switch (c.dtype) {
    case COMPAR_BF16: return run_naive<uint16_t>(c, g, s);
    case COMPAR_F8E4M3: return run_naive<uint8_t>(c, g, s);
    default: return run_naive<float>(c, g, s);
  }
}

int launch_simt(const GemmCall& c, Workspace& ws, const DeviceGuard& g, int num_sms,
                cudaStream_t s) {
  switch (c.dtype) {
    case COMPAR_BF16: return dispatch_simt<uint16_t>(c, ws, g, num_sms, s);
    case COMPAR_F8E4M3: return dispatch_simt<uint8_t>(c, ws, g, num_sms, s);
    default: return dispatch_simt<float>(c, ws, g, num_sms, s);
  }
}

int launch_splitk_reduce(int m, int n, int splits, const float* partial, float alpha, float beta,
                         float* C, int64_t ldc, int num_sms, cudaStream_t s) {
  const int64_t total = static_cast<int64_t>(m) * n;
  if (total <= 0) return COMPAR_OK;
  const int blocks = static_cast<int>(std::min<int64_t>((total + 255) / 256, 4 * num_sms));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  COMPAR_CUDA_TRY(
      cudaLaunchKernelEx(&cfg, splitk_reduce_kernel, m, n, splits, partial, alpha, beta, C, ldc));
  count_launch();
  return COMPAR_OK;
}

int launch_scale_c(float* C, int64_t m, int64_t n, int64_t ldc, float beta, cudaStream_t s) {
  const int64_t total = m * n;
  const int blocks = static_cast<int>(std::min<int64_t>((total + 255) / 256, 4096));
  scale_c_kernel<<<blocks, 256, 0, s>>>(C, static_cast<int>(m), static_cast<int>(n), ldc, beta);
  COMPAR_CUDA_TRY(cudaGetLastError());
  count_launch();
  return COMPAR_OK;
}

// ------------------------------------------------------------------ caller-owned scratch
// The SIMT variant with the same tiles and split-K plan as launch_simt, but
// its split-K partial sums go to `scratch` (capacity `scratch_bytes`), which
// the caller owns; nothing is allocated.  A plan that needs more scratch than
// that is refused with COMPAR_ERR_INVALID and *need_bytes tells how much.
namespace {
template <int BM, int BN, int BK, int TM, int TN>
int run_simt_scratch(const GemmCall& c, float* scratch, size_t scratch_bytes, int num_sms,
                     cudaStream_t s, size_t* need_bytes) {
  const int M = static_cast<int>(c.m), N = static_cast<int>(c.n), K = static_cast<int>(c.k);
  const int tiles_m = (M + BM - 1) / BM, tiles_n = (N + BN - 1) / BN;
  const SimtPlan plan = simt_plan(c, num_sms);
  const int splits = plan.splits, k_per = static_cast<int>(plan.k_per);
  const size_t need = splits > 1 ? static_cast<size_t>(splits) * M * N * sizeof(float) : 0;
  if (need_bytes) *need_bytes = need;
  if (need > scratch_bytes) return COMPAR_ERR_INVALID;
  float* partial = splits > 1 ? scratch : nullptr;
  const bool vec = (c.k % 4 == 0) && (c.n % 4 == 0) && (c.lda % 4 == 0) && (c.ldb % 4 == 0) &&
                   (c.ldc % 4 == 0) && (reinterpret_cast<uintptr_t>(c.A) % 16 == 0) &&
                   (reinterpret_cast<uintptr_t>(c.B) % 16 == 0) &&
                   (reinterpret_cast<uintptr_t>(c.C) % 16 == 0);
  dim3 grid(tiles_n, tiles_m, splits);
  constexpr int threads = SimtCfg<BM, BN, BK, TM, TN, true>::kThreads;
  const float* A = static_cast<const float*>(c.A);
  const float* B = static_cast<const float*>(c.B);
  if (vec)
    gemm_simt_kernel<float, BM, BN, BK, TM, TN, true><<<grid, threads, 0, s>>>(
        M, N, K, k_per, c.alpha, A, c.lda, B, c.ldb, c.beta, c.C, c.ldc, partial);
  else
    gemm_simt_kernel<float, BM, BN, BK, TM, TN, false><<<grid, threads, 0, s>>>(
        M, N, K, k_per, c.alpha, A, c.lda, B, c.ldb, c.beta, c.C, c.ldc, partial);
  COMPAR_CUDA_TRY(cudaGetLastError());
  count_launch();
  if (splits > 1) {
    const int64_t total = static_cast<int64_t>(M) * N;
    const int blocks = static_cast<int>(std::min<int64_t>((total + 255) / 256, 4 * num_sms));
    splitk_reduce_kernel<<<blocks, 256, 0, s>>>(M, N, splits, partial, c.alpha, c.beta, c.C,
                                                c.ldc);
    COMPAR_CUDA_TRY(cudaGetLastError());
    count_launch();
  }
  return COMPAR_OK;
}
}  // namespace

int launch_simt_scratch(const GemmCall& c, float* scratch, size_t scratch_bytes, int num_sms,
                        cudaStream_t s, size_t* need_bytes) {
  const SimtPlan plan = simt_plan(c, num_sms);
  if (plan.skinny) {
    const size_t need =
        plan.splits > 1 ? static_cast<size_t>(plan.splits) * c.m * c.n * sizeof(float) : 0;
    if (need_bytes) *need_bytes = need;
    if (need > scratch_bytes) return COMPAR_ERR_INVALID;
    return run_skinny<float>(c, plan, scratch, nullptr, 0u, num_sms, s);
  }
  if (plan.bm == 32)
    return run_simt_scratch<32, 128, 32, 4, 8>(c, scratch, scratch_bytes, num_sms, s, need_bytes);
  return run_simt_scratch<128, 128, 16, 8, 8>(c, scratch, scratch_bytes, num_sms, s, need_bytes);
}

}  // namespace compar
