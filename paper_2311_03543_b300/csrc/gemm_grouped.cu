// Persistent grouped GEMM: many independent problems of uneven sizes in one
// launch (compar_gemm_batched).  The paper's runtime submits one task per
// call and schedules tasks over processing units (Sec. 2.2); for a batch of
// small GEMMs on one GPU the B300-native form of that is a single persistent
// kernel whose CTAs walk a shared tile list spanning every problem.
//
// Per-problem mode (same stage sizes, chosen per tile at run time):
//   mode 0 BF16   : bf16 operands, one kind::f16 MMA per 32-byte K step
//   mode 1 SPLIT3 : 3xBF16 pieces {hi, lo}, three kind::f16 MMAs per K step
//   mode 2 TF32   : float32 operands, one kind::tf32 MMA per K step
// A is K-major (row-major M x K).  In the bf16 modes B is read as stored,
// K x N with N contiguous (MN-major): TMA boxes of 64 columns x kRow/2 K
// rows, so a bf16 B needs no re-layout at all; TF32 reads a K-major copy.
// Every mode accumulates each chunk of 4 stages in TMEM and adds the chunk
// into FP32 registers (promotion), so no mode carries an accumulation error
// that grows with K.
//
// Problem descriptors (tensor maps, sizes, C, scalars) live in device memory,
// written by the host each call; the operand pre-pass for every problem runs
// as one grouped launch before the GEMM.  Both launches and the descriptor
// upload are captured once per batch shape in a CUDA graph.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "common.h"
#include "epilogue.cuh"
#include "grouped.h"
#include "ptx.cuh"

namespace compar {
namespace {

using dev::Kind;

constexpr int kBM = 128;
constexpr int kRow = kGroupedRow;  // bytes of K per stage and operand row
constexpr int kEpiWarps = 8;  // two per TMEM lane quarter, each half the columns
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kEpi = 32 * kEpiWarps;
constexpr int kMnBox = 64 * kRow;  // one MN-major B box: 64 columns x kRow/2 K rows of bf16
constexpr int kChunkKB = 512 / kRow;  // promotion every 256 bf16 K elements
// The BF16 mode has one piece per operand, so it fills a stage's hi and lo
// regions with one K block of twice the depth: 128-byte rows (128-byte
// swizzle), A as one 128-row box, B as 64-column x 64-row boxes.  A stage
// then carries four MMAs for the same TMA instructions and handshakes, as
// in the single-call BF16 kernel (with 64-byte rows the mode ran at half
// that kernel's rate on the same problem).
constexpr int kRowWide = 2 * kRow;
constexpr int kMnBoxWide = 64 * kRowWide;
__host__ __device__ constexpr int grouped_chunk_kb(int mode) {
  return mode == 0 ? kChunkKB / 2 : kChunkKB;  // K blocks per 256 K elements
}
constexpr int kMaxIndexed = 4096;  // batches up to this size search a shared-memory index

template <int BN>
struct GLayout {
  static constexpr int kA = kBM * kRow;       // one A piece
  static constexpr int kB = BN * kRow;        // one B piece
  static constexpr int kStage = 2 * (kA + kB);
  static constexpr int kBar = 1024;  // barriers, the tile ring, TMEM slot, abort flag
  static constexpr int kIndex = kMaxIndexed * 4;    // problems' tile_start values
  static constexpr int kStagesRaw = (232448 - 1024 - kBar - kIndex) / kStage;
  static constexpr int kStages = kStagesRaw > 6 ? 6 : kStagesRaw;
  static constexpr int kSmem = 1024 + kStages * kStage + kBar + kIndex;
  static constexpr int kTmemCols = 2 * BN < 32 ? 32 : 2 * BN;
};

// Last problem whose first tile is <= tile; s_start holds every problem's
// tile_start in shared memory when the batch has at most kMaxIndexed problems.
__device__ __forceinline__ int find_problem(const GroupProblem* __restrict__ P,
                                            const int* s_start, int count, int tile) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int st = s_start ? s_start[mid] : P[mid].tile_start;
    if (st <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// The fields of a tile's problem that the roles need: the producer looks
// them up once per tile and passes them to the other roles with the tile.
struct TileInfo {
  int q, local, tiles_m, num_kb, mode, M, N;
  float* C;
  int64_t ldc;
  float alpha, beta;
};

__device__ __forceinline__ TileInfo tile_info(const GroupProblem* __restrict__ P,
                                              const int* s_start, int count, int tile) {
  TileInfo t;
  t.q = find_problem(P, s_start, count, tile);
  const GroupProblem& g = P[t.q];
  t.local = tile - (s_start ? s_start[t.q] : g.tile_start);
  t.tiles_m = g.tiles_m;
  t.num_kb = g.num_kb;
  t.mode = g.mode;
  t.M = g.M;
  t.N = g.N;
  t.C = g.C;
  t.ldc = g.ldc;
  t.alpha = g.alpha;
  t.beta = g.beta;
  return t;
}

// Dynamic tile scheduling: the producer takes tile indices from a
// launch-wide counter (zero at launch) and hands each tile, with its
// problem's fields, to the MMA thread and the epilogue warps through a ring
// in shared memory; a CTA that starts late (beside another kernel's CTAs)
// simply takes fewer tiles.  A slot is filled by one arrival and freed by
// the MMA thread and one lane of each epilogue warp once they have read it.
constexpr int kRing = 8;
struct RingTile {
  TileInfo t;
  int tile;  // < 0: no tile left
};

__device__ __forceinline__ bool drain(uint64_t* bar, uint32_t parity, uint64_t budget) {
  const uint64_t t0 = dev::globaltimer_ns();
  while (!dev::mbar_try_wait(bar, parity))
    if (dev::globaltimer_ns() - t0 > budget) return false;
  return true;
}

template <int BN>
__global__ void __maxnreg__(152)
    grouped_gemm_kernel(const GroupProblem* __restrict__ probs, int count, int total_tiles,
                        int* __restrict__ tile_ctr, int* err_word, unsigned long long budget_ns) {
  using L = GLayout<BN>;
  constexpr int S = L::kStages;
  static_assert((2 * S + 5 + 2 * kRing) * 8 + kRing * sizeof(RingTile) + 8 <= L::kBar,
                "barriers and tile ring fit their region");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  // stage s: [A_hi][A_lo][B_hi][B_lo]
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * L::kStage);
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;
  uint64_t* tempty = tfull + 2;
  uint64_t* drainb = tempty + 2;
  uint64_t* ring_full = drainb + 1;     // [kRing]
  uint64_t* ring_empty = ring_full + kRing;
  RingTile* ring = reinterpret_cast<RingTile*>(ring_empty + kRing);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(ring + kRing);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* s_index = reinterpret_cast<int*>(smem + S * L::kStage + L::kBar);
  const int* s_start = count <= kMaxIndexed ? s_index : nullptr;
  if (s_start)
    for (int i = threadIdx.x; i < count; i += blockDim.x) s_index[i] = probs[i].tile_start;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      dev::mbar_init(&full[s], 1);
      dev::mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      dev::mbar_init(&tfull[a], 1);
      dev::mbar_init(&tempty[a], kEpi);
    }
    dev::mbar_init(drainb, 1);
    for (int r = 0; r < kRing; ++r) {
      dev::mbar_init(&ring_full[r], 1);
      dev::mbar_init(&ring_empty[r], 1 + kEpiWarps);
    }
    *abort_flag = 0;
    dev::fence_barrier_init();
  }
  if (warp == 1) {
    dev::tmem_alloc(tmem_slot, L::kTmemCols);
    dev::tmem_relinquish();
  }
  dev::tc_fence_before();
  __syncthreads();
  dev::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const dev::WaitCtx w{abort_flag, err_word, budget_ns};

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------- producer
    uint32_t stage = 0, phase = 0, issued = 0, issued_par = 0;
    bool ok = true;
    // The descriptors were written by the host for this launch; earlier
    // launches may have left other bytes at these addresses in the cache:
    // acquire (and prefetch) a problem's maps before its first TMA use.
    auto acquire_maps = [&](int q) {
      const GroupProblem& P = probs[q];
      dev::tensormap_acquire(&P.map_a);
      dev::tensormap_acquire(&P.map_b);
      dev::tensormap_acquire(&P.map_a2);
      dev::tensormap_acquire(&P.map_b2);
      dev::tma_prefetch_desc(&P.map_a);
      dev::tma_prefetch_desc(&P.map_b);
    };
    int next = atomicAdd(tile_ctr, 1);
    int last_q = -1;
    for (int i = 0; ok; ++i) {
      const int tile = next < total_tiles ? next : -1;
      // the following tile's index is in flight while this tile loads
      if (tile >= 0) next = atomicAdd(tile_ctr, 1);
      const int slot = i % kRing;
      if (!dev::mbar_wait(&ring_empty[slot], ((i / kRing) & 1) ^ 1, w)) {
        ok = false;
        break;
      }
      TileInfo cur{};
      if (tile >= 0) cur = tile_info(probs, s_start, count, tile);
      ring[slot].t = cur;
      ring[slot].tile = tile;
      dev::mbar_arrive(&ring_full[slot]);
      if (tile < 0) break;
      if (cur.q != last_q) {
        acquire_maps(cur.q);
        last_q = cur.q;
      }
      const GroupProblem& P = probs[cur.q];
      const int mb = cur.local % cur.tiles_m, nb = cur.local / cur.tiles_m;
      const bool wide = cur.mode == 0;  // one deep K block fills the stage
      const int pieces = cur.mode == 1 ? 2 : 1;
      const uint32_t tx = static_cast<uint32_t>((wide ? 2 : pieces) * (L::kA + L::kB));
      const bool tf32 = cur.mode == 2;
      const int kelems = tf32 ? kRow / 4 : (wide ? kRowWide / 2 : kRow / 2);
      const int num_kb = cur.num_kb;
      for (int kb = 0; kb < num_kb; ++kb) {
        if (!dev::mbar_wait(&empty[stage], phase ^ 1, w)) {
          ok = false;
          break;
        }
        dev::mbar_arrive_expect_tx(&full[stage], tx);
        uint8_t* st = smem + stage * L::kStage;
        const int x = kb * kelems;
        dev::tma_load_2d(st, &P.map_a, &full[stage], x, mb * kBM);
        if (pieces == 2) dev::tma_load_2d(st + L::kA, &P.map_a2, &full[stage], x, mb * kBM);
        if (tf32) {
          dev::tma_load_2d(st + 2 * L::kA, &P.map_b, &full[stage], x, nb * BN);
        } else if (wide) {
#pragma unroll
          for (int h = 0; h < BN / 64; ++h)
            dev::tma_load_2d(st + 2 * L::kA + h * kMnBoxWide, &P.map_b, &full[stage],
                             nb * BN + h * 64, x);
        } else {
#pragma unroll
          for (int h = 0; h < BN / 64; ++h) {
            dev::tma_load_2d(st + 2 * L::kA + h * kMnBox, &P.map_b, &full[stage],
                             nb * BN + h * 64, x);
            if (pieces == 2)
              dev::tma_load_2d(st + 2 * L::kA + L::kB + h * kMnBox, &P.map_b2, &full[stage],
                               nb * BN + h * 64, x);
          }
        }
        issued |= 1u << stage;
        issued_par = (issued_par & ~(1u << stage)) | (phase << stage);
        if (++stage == S) {
          stage = 0;
          phase ^= 1;
        }
      }
    }
    if (!ok)
      for (int s = 0; s < S; ++s)
        if (issued & (1u << s)) drain(&full[s], (issued_par >> s) & 1, budget_ns);
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------- MMA issuer
    constexpr uint32_t id_f16 = dev::make_idesc_bmn(1, 1, kBM, BN);
    constexpr uint32_t id_tf32 = dev::make_idesc(2, 2, kBM, BN);
    uint32_t stage = 0, phase = 0;
    int acc_iter = 0;
    bool ok = true;
    for (int i = 0; ok; ++i) {
      const int slot = i % kRing;
      if (!dev::mbar_wait(&ring_full[slot], (i / kRing) & 1, w)) {
        ok = false;
        break;
      }
      const int tile = ring[slot].tile;
      const int mode = ring[slot].t.mode;
      const int num_kb = ring[slot].t.num_kb;
      dev::mbar_arrive(&ring_empty[slot]);
      if (tile < 0) break;
      const int ckb = grouped_chunk_kb(mode);
      for (int kb0 = 0; ok && kb0 < num_kb; kb0 += ckb, ++acc_iter) {
        const uint32_t acc = acc_iter & 1, acc_phase = (acc_iter >> 1) & 1;
        if (!dev::mbar_wait(&tempty[acc], acc_phase ^ 1, w)) {
          ok = false;
          break;
        }
        dev::tc_fence_after();
        const uint32_t d = tmem_base + acc * BN;
        const int kb_end = min(num_kb, kb0 + ckb);
        for (int kb = kb0; kb < kb_end; ++kb) {
          if (!dev::mbar_wait(&full[stage], phase, w)) {
            ok = false;
            break;
          }
          dev::tc_fence_after();
          const uint32_t s0 = dev::smem_u32(smem + stage * L::kStage);
          if (mode == 0) {
            // one 64-deep K block: A K-major in 128-byte rows, B MN-major in
            // 64-column x 64-row boxes; four MMAs of 16 K rows
            const uint64_t dw = dev::smem_desc_kmajor<kRowWide>(s0);
#pragma unroll
            for (int kk = 0; kk < kRowWide / 32; ++kk) {
              const uint64_t ko = static_cast<uint64_t>(kk * 32) >> 4;
              const uint64_t db =
                  dev::smem_desc_sw128_mnmajor(s0 + 2 * L::kA + kk * 2048, kMnBoxWide);
              dev::mma<Kind::F16>(d, dw + ko, db, id_f16, (kb == kb0 && kk == 0) ? 0u : 1u);
            }
            dev::mma_commit(&empty[stage]);
            if (++stage == S) {
              stage = 0;
              phase ^= 1;
            }
            continue;
          }
          const uint64_t da = dev::smem_desc_kmajor<kRow>(s0);
          const uint64_t da2 = dev::smem_desc_kmajor<kRow>(s0 + L::kA);
#pragma unroll
          for (int kk = 0; kk < kRow / 32; ++kk) {
            // A: 32 bytes of K per instruction inside the swizzled row
            const uint64_t ko = static_cast<uint64_t>(kk * 32) >> 4;
            const uint32_t first = (kb == kb0 && kk == 0) ? 0u : 1u;
            if (mode == 2) {
              const uint64_t db = dev::smem_desc_kmajor<kRow>(s0 + 2 * L::kA);
              dev::mma<Kind::TF32>(d, da + ko, db + ko, id_tf32, first);
            } else {
              // 3xBF16; B (MN-major): 16 K rows per instruction, 2048 bytes
              const uint32_t bk = s0 + 2 * L::kA + kk * 2048;
              const uint64_t db = dev::smem_desc_sw128_mnmajor(bk, kMnBox);
              const uint64_t db2 = dev::smem_desc_sw128_mnmajor(bk + L::kB, kMnBox);
              dev::mma<Kind::F16>(d, da + ko, db, id_f16, first);
              dev::mma<Kind::F16>(d, da + ko, db2, id_f16, 1u);
              dev::mma<Kind::F16>(d, da2 + ko, db, id_f16, 1u);
            }
          }
          dev::mma_commit(&empty[stage]);
          if (++stage == S) {
            stage = 0;
            phase ^= 1;
          }
        }
        if (!ok) break;
        dev::mma_commit(&tfull[acc]);
      }
    }
    dev::mma_commit(drainb);
    drain(drainb, 0, budget_ns);
  } else if (warp >= 2) {
    // ---------------------------------------------------------- epilogue
    // Warp w reads TMEM lane quarter w % 4 (the hardware's access rule) and
    // one half of the columns.
    constexpr int EC = BN / 2;       // columns of this warp's slice
    constexpr int J = EC / 8;        // 16x256b repetitions per fragment
    static_assert(J == 4 || J == 8 || J == 16, "epilogue slice of 32, 64 or 128 columns");
    const int quarter = warp & 3;
    const int cslice = (warp - 2) / 4;
    int acc_iter = 0;
    bool ok = true;
    for (int i = 0; ok; ++i) {
      const int slot = i % kRing;
      if (!dev::mbar_wait(&ring_full[slot], (i / kRing) & 1, w)) {
        ok = false;
        break;
      }
      const int tile = ring[slot].tile;
      const TileInfo t = ring[slot].t;
      __syncwarp();
      if (lane == 0) dev::mbar_arrive(&ring_empty[slot]);
      if (tile < 0) break;
      const int mb = t.local % t.tiles_m, nb = t.local / t.tiles_m;
      const int pM = t.M, pN = t.N, num_kb = t.num_kb;
      float* const pC = t.C;
      const int64_t ldc = t.ldc;
      const float alpha = t.alpha, beta = t.beta;
      // two 16-row fragments (row halves of the warp's lane quarter)
      float sum[2][4 * J];
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < 4 * J; ++j) sum[h][j] = 0.f;
      const int ckb = grouped_chunk_kb(t.mode);
      const int chunks = (num_kb + ckb - 1) / ckb;
      for (int ch = 0; ch < chunks; ++ch, ++acc_iter) {
        const uint32_t acc = acc_iter & 1, acc_phase = (acc_iter >> 1) & 1;
        if (!dev::mbar_wait(&tfull[acc], acc_phase, w)) {
          ok = false;
          break;
        }
        dev::tc_fence_after();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint32_t taddr = tmem_base +
                                 (static_cast<uint32_t>(quarter * 32 + 16 * h) << 16) +
                                 acc * BN + cslice * EC;
          if constexpr (J == 16) {
            // two 64-column loads: repetitions 0-7 and 8-15 of the fragment
#pragma unroll
            for (int half = 0; half < 2; ++half) {
              uint32_t r[32];
              dev::tmem_ld_16x256b_x8(taddr + 64 * half, r);
              dev::tmem_ld_wait();
#pragma unroll
              for (int j = 0; j < 32; ++j) sum[h][32 * half + j] += __uint_as_float(r[j]);
            }
          } else {
            uint32_t r[4 * J];
            if constexpr (J == 8) dev::tmem_ld_16x256b_x8(taddr, r);
            else dev::tmem_ld_16x256b_x4(taddr, r);
            dev::tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 4 * J; ++j) sum[h][j] += __uint_as_float(r[j]);
          }
        }
        dev::tc_fence_before();
        dev::mbar_arrive(&tempty[acc]);
      }
      if (!ok) break;
      // Sector-wide stores straight from the fragments; warps whose rows or
      // columns lie wholly outside the problem store nothing.
      const int row0 = mb * kBM + quarter * 32;
      const int col0 = nb * BN + cslice * EC;
      if (row0 >= pM || col0 >= pN) continue;
      const bool vec2 = (ldc % 2 == 0) && ((reinterpret_cast<uintptr_t>(pC) & 7) == 0);
#pragma unroll
      for (int h = 0; h < 2; ++h)
        store_frag<J>(sum[h], pC, ldc, pM, pN, row0 + 16 * h, col0, alpha, beta, vec2, lane);
    }
  }
  __syncthreads();
  if (warp == 1) {
    dev::tc_fence_after();
    dev::tmem_dealloc(tmem_base, L::kTmemCols);
  }
}

}  // namespace

int grouped_smem_bytes(int bn) {
  return bn == 256 ? GLayout<256>::kSmem : GLayout<128>::kSmem;
}

int launch_grouped_gemm(int bn, const GroupProblem* d_probs, int count, int total_tiles,
                        int* d_tile_ctr, const DeviceGuard& g, int num_sms, cudaStream_t s) {
  if (count <= 0 || total_tiles <= 0) return COMPAR_OK;
  if (d_tile_ctr == nullptr) return COMPAR_ERR_INVALID;
  // the launch's tile counter starts from zero (a memset node in a graph)
  COMPAR_CUDA_TRY(cudaMemsetAsync(d_tile_ctr, 0, sizeof(int), s));
  const int grid = std::min(total_tiles, num_sms);
  if (bn == 256) {
    COMPAR_CUDA_TRY(smem_opt_in(reinterpret_cast<const void*>(grouped_gemm_kernel<256>),
                                GLayout<256>::kSmem));
    grouped_gemm_kernel<256><<<grid, kThreads, GLayout<256>::kSmem, s>>>(
        d_probs, count, total_tiles, d_tile_ctr, g.err_word, g.budget_ns);
  } else {
    COMPAR_CUDA_TRY(smem_opt_in(reinterpret_cast<const void*>(grouped_gemm_kernel<128>),
                                GLayout<128>::kSmem));
    grouped_gemm_kernel<128><<<grid, kThreads, GLayout<128>::kSmem, s>>>(
        d_probs, count, total_tiles, d_tile_ctr, g.err_word, g.budget_ns);
  }
  COMPAR_CUDA_TRY(cudaGetLastError());
  count_launch();
  return COMPAR_OK;
}

}  // namespace compar
