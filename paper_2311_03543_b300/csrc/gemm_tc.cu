// Tensor-core implementation variants of C = alpha*A*B + beta*C on sm_103a
// (the matrix-multiply component of Sec. 2.1 / Table 2; the paper's GPU
// variants were SIMT CUDA and cuBLAS on a Pascal GPU without tensor cores).
//
// One persistent, warp-specialised kernel template serves four variants:
//   TF32   : kind::tf32 on float32 operands (tensor cores read 19 bits)
//   BF16   : kind::f16 with bf16 operands
//   FP8    : kind::f8f6f4 with E4M3 operands, per-tensor dequantisation
//   SPLIT3 : 3xBF16 — A = Ahi + Alo, B = Bhi + Blo (bf16 pieces) and
//            Ahi*Bhi + Ahi*Blo + Alo*Bhi accumulated into one FP32 TMEM tile
//   SPLIT3_TF32 : 3xTF32 — A = Ahi + Alo, B = Bhi + Blo (TF32 pieces, kept
//            in float32) and the three products on kind::tf32, the two small
//            ones first, promoted after every stage
//   SPLIT3_FUSED : 3xBF16 on float32 A and B read by TMA as they are; the
//            epilogue warps split every stage in shared memory, in place
//            (hi and lo 512-byte atoms interleaved), between promotions
//   SPLIT6 : 3-piece split A = Ah + Am + Al (likewise B) and the six products
//            whose size is at least 2^-16 of Ah*Bh: Ah*Bm, Am*Bh, Ah*Bl,
//            Am*Bm, Al*Bh first, Ah*Bh last, promoted into FP32 registers
//            after every stage
//
// CTA roles (one CTA per SM, grid = min(tiles, SMs)):
//   warp 0      TMA producer: one elected lane streams K-major A and B tiles
//               (128- or 64-byte swizzle) into an S-stage shared-memory ring.
//   warp 1      TMEM allocator; one lane issues tcgen05.mma into one of two
//               TMEM accumulators (double buffered across output tiles or
//               K chunks) and releases ring stages with tcgen05.commit.
//   warps 2..   epilogue (4 or 8 warps): tcgen05.ld (16x256b fragments) of
//               the accumulator lane quarter the warp may access (and its
//               column slice), alpha/beta and dequantisation, sector-wide
//               float2 stores to C.
// Every wait is bounded (ptx.cuh); on expiry the CTA drains its own copies
// and MMAs, frees TMEM and returns with COMPAR_ERR_TIMEOUT in the error word.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cooperative_groups.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <type_traits>

#include "common.h"
#include "epilogue.cuh"
#include "ptx.cuh"

namespace compar {
namespace {

using dev::Kind;

constexpr int kBM = 128;

// Per-variant geometry: `row` = bytes of K per stage and operand row (128 or
// 64, the TMA / MMA swizzle width), `epi` = epilogue warps (each lane quarter
// of the accumulator is read by epi/4 warps, each taking BN*4/epi columns),
// `chunk_kb` = stages per promoted K chunk (0: no promotion).
template <int V>
struct Traits;
template <>
struct Traits<COMPAR_V_TC_TF32> {
  static constexpr Kind kind = Kind::TF32;
  static constexpr int elem = 4, fmt = 2, pieces = 1, BN = 256, row = 128, chunk_kb = 0, epi = 4;
  static constexpr bool b_mn = false, small_first = false, fused = false;
};
// 3xTF32: float32 pieces, 64-byte rows (16 K elements per 48 KB stage); each
// stage is a promoted chunk with the two small products issued first, so
// the truncating accumulator adds the leading product once per K step onto
// a partial 2^-11 its size.
template <>
struct Traits<COMPAR_V_SPLIT3_TF32> {
  static constexpr Kind kind = Kind::TF32;
  static constexpr int elem = 4, fmt = 2, pieces = 2, BN = 256, row = 64, chunk_kb = 1, epi = 8;
  static constexpr bool b_mn = false, small_first = true, fused = false;
};
template <>
struct Traits<COMPAR_V_TC_BF16> {
  static constexpr Kind kind = Kind::F16;
  static constexpr int elem = 2, fmt = 1, pieces = 1, BN = 256, row = 128, chunk_kb = 0, epi = 4;
  static constexpr bool b_mn = true, small_first = false, fused = false;
};
template <>
struct Traits<COMPAR_V_TC_FP8> {
  static constexpr Kind kind = Kind::F8;
  static constexpr int elem = 1, fmt = 0, pieces = 1, BN = 256, row = 128, chunk_kb = 0, epi = 4;
  static constexpr bool b_mn = false, small_first = false, fused = false;
};
// 3xBF16: 64-byte rows give 48 KB stages (four of them) for a 128 x 256 tile;
// promotion every 8 stages = 256 K elements.
template <>
struct Traits<COMPAR_V_SPLIT3> {
  static constexpr Kind kind = Kind::F16;
  static constexpr int elem = 2, fmt = 1, pieces = 2, BN = 256, row = 64, chunk_kb = 8, epi = 8;
  static constexpr bool b_mn = true, small_first = false, fused = false;
};
// Fused 3xBF16: a stage holds the float32 A tile (128 rows x 32 K, 16 KB)
// and B tile (32 K x 256 N in 16 boxes of 64 N x 8 K, 32 KB) as TMA wrote
// them; the split overwrites each with its bf16 hi and lo pieces, which take
// the same bytes, so the ring keeps the four 48 KB stages of SPLIT3.  A
// becomes K-major, B stays MN-major (as stored, no transpose).  (Sixteen
// epilogue warps with 64 sums each were slower: 96 registers a thread.)
template <>
struct Traits<COMPAR_V_SPLIT3_FUSED> {
  static constexpr Kind kind = Kind::F16;
  static constexpr int elem = 2, fmt = 1, pieces = 2, BN = 256, row = 64, chunk_kb = 8, epi = 8;
  static constexpr bool b_mn = true, small_first = false, fused = true;
};
// 6-product split: three pieces per operand make 72 KB stages (three of
// them).  Each stage is its own promoted chunk: within it the five small
// products are summed first, so the tensor core's truncating accumulator
// adds the leading product once per K step onto a partial 2^-8 its size.
template <>
struct Traits<COMPAR_V_SPLIT6> {
  static constexpr Kind kind = Kind::F16;
  static constexpr int elem = 2, fmt = 1, pieces = 3, BN = 256, row = 64, chunk_kb = 1, epi = 8;
  static constexpr bool b_mn = false, small_first = true, fused = false;
};

// kPair: the tile is computed by a CTA pair (cta_group::2): 2 kBM rows x BN,
// each CTA holding its kBM rows of A and BN / 2 rows (columns) of B in its
// shared memory and its kBM rows of the accumulator in its tensor memory.
template <int V, bool kPair = false>
struct Layout {
  using T = Traits<V>;
  static constexpr int BN = T::BN;
  static constexpr int kBRows = kPair ? BN / 2 : BN;  // rows of B this CTA loads
  static constexpr int kABytes = kBM * T::row;
  static constexpr int kBBytes = kBRows * T::row;
  static constexpr int kStageBytes = T::pieces * (kABytes + kBBytes);
  static constexpr int kMaxSmem = 232448;  // 227 KB opt-in per CTA
  static constexpr int kBarBytes = 256;
  static constexpr int kStagesRaw = (kMaxSmem - 1024 - kBarBytes) / kStageBytes;
  static constexpr int kStages = kStagesRaw > 6 ? 6 : kStagesRaw;
  static constexpr int kRingBytes = kStages * kStageBytes;
  // TMA-store epilogue: two 2 KB staging boxes per epilogue warp, where the
  // ring leaves room for them
  static constexpr int kEpiWarpBytes = 2 * 2048;
  static constexpr bool kTmaStore =
      1024 + kRingBytes + T::epi * kEpiWarpBytes + kBarBytes <= kMaxSmem;
  static constexpr int kEpiStageBytes = kTmaStore ? T::epi * kEpiWarpBytes : 0;
  static constexpr int kSmemBytes = 1024 + kRingBytes + kEpiStageBytes + kBarBytes;
  static constexpr int kTmemCols = 2 * BN;  // two accumulators
  static constexpr int kElemsPerStage = T::row / T::elem;
  // MN-major B (16-bit types): boxes of 64 columns x kElemsPerStage K rows,
  // 128-byte rows, one per 64 columns of the tile
  static constexpr int kMnBox = 64 * 2 * kElemsPerStage;
  static_assert(kMnBox % 1024 == 0, "MN-major boxes hold whole 8-row swizzle groups");
  static constexpr int kMmaM = kPair ? 2 * kBM : kBM;  // rows of one MMA
  // arrivals that free an accumulator: every epilogue thread, or in a pair
  // one elected lane per epilogue warp of both CTAs (on the even CTA's barrier)
  static constexpr int kTemptyCount = kPair ? 2 * T::epi : 32 * T::epi;
  static constexpr int kThreads = 64 + 32 * T::epi;
  static constexpr int kEpiThreads = 32 * T::epi;
  static constexpr int kEpiCols = BN * 4 / T::epi;  // columns one epilogue warp handles
  static_assert(kStages >= 2, "pipeline needs two stages");
  static_assert(kPair || kStages * kStageBytes >= kBM * BN * 4,
                "an in-cluster K split stages a kBM x BN float tile in the ring");
  static_assert(kTmemCols <= 512 && (kTmemCols & (kTmemCols - 1)) == 0, "TMEM columns");
  static_assert(T::epi % 4 == 0 && kEpiCols % 32 == 0, "epilogue split");
};

struct TcArgs {
  int M, N, K;
  int num_kb;
  int tiles_m, tiles_n;
  // Split K (few tiles, long K): work unit u = tile u / splits, K blocks
  // [(u % splits) * kb_per_split, +kb_per_split).  With split_cluster the
  // splits of a tile are one thread-block cluster (split = rank in it) that
  // adds its accumulators through distributed shared memory; otherwise each
  // unit writes alpha * partial to partial[split][M][N] and a reduce kernel
  // forms C.
  int splits, kb_per_split;
  int split_cluster;
  float* partial;
  // Work list of a CTA: the `dp_units` classic units (whole tiles, or tile x
  // K-split units when splits > 1) dealt round-robin, then, when sk_q > 0, a
  // stream-K tail: tiles sk_tile0.. are cut into promotion chunks (sk_cpt
  // per tile, sk_q in all) and CTA b < sk_ctas takes the contiguous chunks
  // [b sk_q / sk_ctas, (b+1) sk_q / sk_ctas), at most two pieces of tiles.
  int dp_units;
  int sk_tile0, sk_cpt, sk_q, sk_ctas;
  float* sk_slab;               // [sk_ctas * pair][2][kBM * BN] published pieces
  // [tail tiles * pair] arrival words: (epoch << 32 | count), a word with
  // another launch's epoch counting as zero (no reset between calls)
  unsigned long long* sk_count;
  unsigned int sk_epoch;
  // 1, or 2 when CTA pairs compute the tiles: a "CTA" of the work list
  // (blockIdx.x / pair) is then a pair, a tile is 2 kBM x BN, and each CTA
  // of the pair publishes and counts its own kBM rows of a stream-K tile.
  int pair;
  // 1: whole-tile stores of C go through the TMA-store epilogue (beta == 0,
  // no K split, C rows 16-byte aligned)
  int tma_c;
  float alpha, beta;
  const float* dequant_a;  // optional device factors (fp8 of float32 inputs)
  const float* dequant_b;
  float* C;
  int64_t ldc;
  int* err_word;
  unsigned long long budget_ns;
};

__device__ __forceinline__ void tile_coords(int tile, int tiles_m, int tiles_n, int& mb, int& nb) {
  constexpr int G = 8;  // group of M blocks walked together for L2 reuse of B
  const int per_group = G * tiles_n;
  const int group = tile / per_group;
  const int first_m = group * G;
  const int gsize = min(tiles_m - first_m, G);
  const int in = tile - group * per_group;
  mb = first_m + in % gsize;
  nb = in / gsize;
}

// One item of a CTA's work list: K blocks [kb_begin, kb_end) of a tile.
// piece = -1: a classic unit (split = its K-split index); piece 0 / 1: the
// first / second stream-K piece of this CTA.
struct WorkItem {
  int tile, kb_begin, kb_end, split, piece;
};

__device__ __forceinline__ int sk_start(const TcArgs& p, int b) {
  return static_cast<int>(static_cast<long long>(b) * p.sk_q / p.sk_ctas);
}
// The stream-K CTA whose chunk range holds chunk q (ranges are never empty).
__device__ __forceinline__ int sk_cta_of(const TcArgs& p, int q) {
  return static_cast<int>((static_cast<long long>(q + 1) * p.sk_ctas - 1) / p.sk_q);
}

// K blocks per stream-K chunk of the variants without promotion (their
// accumulator spans the whole piece); promoted variants use their chunk.
constexpr int kPlainSkChunk = 2;

// Item i of this CTA's list; false past its end.  Every role of the CTA
// walks the same list.
template <int kChunkKB>
__device__ __forceinline__ bool get_item(const TcArgs& p, int i, WorkItem& it) {
  constexpr int kSk = kChunkKB > 0 ? kChunkKB : kPlainSkChunk;
  const int b = blockIdx.x / p.pair, grid = gridDim.x / p.pair;
  const int u = b + i * grid;
  if (u < p.dp_units) {
    it.tile = u / p.splits;
    it.split = u % p.splits;
    it.kb_begin = it.split * p.kb_per_split;
    it.kb_end = min(p.num_kb, it.kb_begin + p.kb_per_split);
    it.piece = -1;
    return true;
  }
  if (p.sk_q == 0 || b >= p.sk_ctas) return false;
  const int n_dp = b < p.dp_units ? (p.dp_units - 1 - b) / grid + 1 : 0;
  const int k = i - n_dp;
  const int q0 = sk_start(p, b), q1 = sk_start(p, b + 1);
  const int q = k == 0 ? q0 : (q0 / p.sk_cpt + 1) * p.sk_cpt;
  if (k > 1 || q >= q1) return false;
  const int t = q / p.sk_cpt;
  const int qe = min(q1, (t + 1) * p.sk_cpt);
  it.tile = p.sk_tile0 + t;
  it.split = 0;
  it.kb_begin = (q - t * p.sk_cpt) * kSk;
  it.kb_end = min(p.num_kb, (qe - t * p.sk_cpt) * kSk);
  it.piece = k;
  return true;
}

// Wait that ignores the CTA abort flag: used only to drain this CTA's own
// outstanding copies / MMAs before it frees resources and exits.
__device__ __forceinline__ bool drain_wait(uint64_t* bar, uint32_t parity, uint64_t budget) {
  const uint64_t t0 = dev::globaltimer_ns();
  while (!dev::mbar_try_wait(bar, parity)) {
    if (dev::globaltimer_ns() - t0 > budget) return false;
  }
  return true;
}

// ------------------------------------------------------------------ in-place split
// bf16 pieces of a float4: hi = bf16(x) (round to nearest even), lo =
// bf16(x - hi) (the residual is exact in float32), packed low element first.
__device__ __forceinline__ uint32_t bf16x2_bits(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ void split4(const float4 v, uint2& hi, uint2& lo) {
  hi.x = bf16x2_bits(v.x, v.y);
  hi.y = bf16x2_bits(v.z, v.w);
  // the hi values as float32: the bf16 bits in the upper half
  const float hx = __uint_as_float(hi.x << 16), hy = __uint_as_float(hi.x & 0xFFFF0000u);
  const float hz = __uint_as_float(hi.y << 16), hw = __uint_as_float(hi.y & 0xFFFF0000u);
  lo.x = bf16x2_bits(v.x - hx, v.y - hy);
  lo.y = bf16x2_bits(v.z - hz, v.w - hw);
}

// Splits one stage of the fused 3xBF16 variant in place.  As TMA wrote it,
// A is [128 rows][32 K] float32 (128-byte rows) and B is 16 boxes of
// [8 K][64 N] float32 (256-byte rows; box (ng, kg) at 2048 (4 ng + kg)).
// Afterwards every A region of 1024 bytes holds an 8-row atom of the hi
// piece (+0) and of the lo piece (+512), K-major with the 64-byte swizzle
// (16-byte chunk c of row r at c ^ ((r >> 1) & 3)); every B box holds an
// 8-K-row atom of hi (+0) and lo (+1024), MN-major with the 128-byte swizzle
// (chunk c of K row k at c ^ k).  Each region is read whole by one warp
// before that warp writes it (warp cw of kWarps: kPer = 16 / kWarps A row
// groups and B boxes from kPer cw on), so no other warp's data is
// overwritten.  Loads and stores are bank-conflict free.
template <int kWarps>
__device__ __forceinline__ void split_stage_in_place(uint8_t* a_st, uint8_t* b_st, int cw,
                                                     int lane) {
  static_assert(kWarps == 8 || kWarps == 16, "16 A row groups and 16 B boxes per stage");
  constexpr int kPer = 16 / kWarps;  // A groups and B boxes per warp
  {
    // A: lane = (row r of the 8-row group, 32-byte quarter q of the row)
    const int r = lane >> 2, q = lane & 3, h0 = r & 1;
    const int off = 64 * r + 16 * (q ^ ((r >> 1) & 3));
#pragma unroll
    for (int gi = 0; gi < kPer; ++gi) {
      uint8_t* g = a_st + 1024 * (kPer * cw + gi);
      const float4 u = *reinterpret_cast<const float4*>(g + 128 * r + 32 * q + 16 * h0);
      const float4 v = *reinterpret_cast<const float4*>(g + 128 * r + 32 * q + 16 * (h0 ^ 1));
      __syncwarp();
      uint2 h1, l1, h2, l2;
      split4(h0 ? v : u, h1, l1);  // elements 8q..8q+3
      split4(h0 ? u : v, h2, l2);  // elements 8q+4..8q+7
      *reinterpret_cast<uint4*>(g + off) = make_uint4(h1.x, h1.y, h2.x, h2.y);
      *reinterpret_cast<uint4*>(g + 512 + off) = make_uint4(l1.x, l1.y, l2.x, l2.y);
    }
  }
#pragma unroll
  for (int bi = 0; bi < kPer; ++bi) {
    // B: load i gives lane the float4 (N 4c..4c+3) of K row k = 2i + lane/16
    uint8_t* box = b_st + 2048 * (kPer * cw + bi);
    const int c = lane & 15, kh = lane >> 4;
    float4 v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
      v[i] = *reinterpret_cast<const float4*>(box + 256 * (2 * i + kh) + 16 * c);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = 2 * i + kh;
      const int off = 128 * k + 16 * ((c >> 1) ^ k) + 8 * (c & 1);
      uint2 hi, lo;
      split4(v[i], hi, lo);
      *reinterpret_cast<uint2*>(box + off) = hi;
      *reinterpret_cast<uint2*>(box + 1024 + off) = lo;
    }
  }
}

// Stream-K piece bookkeeping: the piece's tail tile t, the tile's first
// chunk, its first contributing CTA b0 and the number of contributors nc.
struct SkPiece {
  int t, first, b0, nc;
};
__device__ __forceinline__ SkPiece sk_piece(const TcArgs& p, const WorkItem& it) {
  SkPiece sp{0, 0, 0, 1};
  if (it.piece < 0) return sp;
  sp.t = it.tile - p.sk_tile0;
  sp.first = sp.t * p.sk_cpt;
  sp.b0 = sk_cta_of(p, sp.first);
  sp.nc = sk_cta_of(p, sp.first + p.sk_cpt - 1) - sp.b0 + 1;
  return sp;
}

// Published partial tile of CTA `cta`'s piece k: kBM x BN floats as float4,
// element (f * 8 + j4) * kEpiThreads + epilogue thread.
template <int BN>
__device__ __forceinline__ float4* sk_slab(const TcArgs& p, int cta, int k) {
  constexpr int64_t kSlab = static_cast<int64_t>(kBM) * BN / 4;
  return reinterpret_cast<float4*>(p.sk_slab) + (2 * static_cast<int64_t>(cta) + k) * kSlab;
}

// After this CTA has published its piece of a tile with several
// contributors: count it in, and if it arrived last add the pieces in
// contributor order (so the result does not depend on which CTA finished
// last) and store the tile.  No CTA waits for another.  False when a bounded
// wait gave up.
template <int NF, int kEpiThreads, int BN>
__device__ __forceinline__ bool sk_count_and_sum(const TcArgs& p, const SkPiece& sp,
                                                 uint64_t* epi_bar, uint32_t& epi_uses,
                                                 volatile int* last_flag, const dev::WaitCtx& w,
                                                 int etid, int lane, float* out, int64_t out_ld,
                                                 int row_q, int col_s, float alpha, float beta,
                                                 bool vec_out) {
  __threadfence();
  // bounded rendezvous: a CTA that gave up elsewhere cannot hang here
  dev::mbar_arrive(epi_bar);
  if (!dev::mbar_wait(epi_bar, epi_uses++ & 1, w)) return false;
  if (etid == 0) {
    __threadfence();
    // in a CTA pair each CTA counts (and sums) its own rows of the tile
    unsigned long long* cnt =
        p.sk_count + sp.t * p.pair + static_cast<int>(blockIdx.x) % p.pair;
    unsigned long long seen = *reinterpret_cast<volatile unsigned long long*>(cnt);
    unsigned int before;
    for (;;) {  // at most nc contributors contend for one word
      before = static_cast<unsigned int>(seen >> 32) == p.sk_epoch ? static_cast<unsigned int>(seen)
                                                                  : 0u;
      const unsigned long long next =
          (static_cast<unsigned long long>(p.sk_epoch) << 32) | (before + 1u);
      const unsigned long long got = atomicCAS(cnt, seen, next);
      if (got == seen) break;
      seen = got;
    }
    *last_flag = before == static_cast<unsigned int>(sp.nc - 1);
  }
  dev::mbar_arrive(epi_bar);
  if (!dev::mbar_wait(epi_bar, epi_uses++ & 1, w)) return false;
  if (!*last_flag) return true;
  __threadfence();
  // the pieces in contributor order, this CTA's own from its slab too; the
  // slabs of contributor b (a pair when p.pair == 2) are those of its CTA
  // b * pair + rank
  const int k0 = sk_start(p, sp.b0) < sp.first ? 1 : 0;  // b0's piece of this tile
  const int rank = static_cast<int>(blockIdx.x) % p.pair;
  if (row_q < p.M && col_s < p.N) {
    // G fragments at a time (8 G independent loads in flight per
    // contributor), so a tile costs NF / G * nc L2 round trips; G = 1 when
    // the epilogue warps have few registers
    constexpr int G = NF >= 4 ? 2 : 1;
    static_assert(NF % G == 0, "fragment groups");
#pragma unroll 1
    for (int f0 = 0; f0 < NF; f0 += G) {
      const int64_t base = f0 * 8 * kEpiThreads + etid;
      float4 acc[8 * G];
      const float4* s0 = sk_slab<BN>(p, sp.b0 * p.pair + rank, k0) + base;
#pragma unroll
      for (int e = 0; e < 8 * G; ++e) acc[e] = __ldcg(s0 + e * kEpiThreads);
      for (int jj = 1; jj < sp.nc; ++jj) {
        const float4* sj = sk_slab<BN>(p, (sp.b0 + jj) * p.pair + rank, 0) + base;
        float4 c[8 * G];
#pragma unroll
        for (int e = 0; e < 8 * G; ++e) c[e] = __ldcg(sj + e * kEpiThreads);
#pragma unroll
        for (int e = 0; e < 8 * G; ++e) {
          acc[e].x += c[e].x;
          acc[e].y += c[e].y;
          acc[e].z += c[e].z;
          acc[e].w += c[e].w;
        }
      }
#pragma unroll
      for (int h = 0; h < G; ++h) {
        float v[32];
#pragma unroll
        for (int j4 = 0; j4 < 8; ++j4) {
          v[4 * j4] = acc[8 * h + j4].x;
          v[4 * j4 + 1] = acc[8 * h + j4].y;
          v[4 * j4 + 2] = acc[8 * h + j4].z;
          v[4 * j4 + 3] = acc[8 * h + j4].w;
        }
        const int f = f0 + h;
        store_frag<8>(v, out, out_ld, p.M, p.N, row_q + 16 * (f & 1), col_s + 64 * (f >> 1),
                      alpha, beta, vec_out, lane);
      }
    }
  }
  return true;
}

// ------------------------------------------------------------------ in-cluster split K
// The kernel's shared-memory ring: dynamic shared memory rounded up to 1 KB.
__device__ __forceinline__ uint8_t* ring_base() {
  extern __shared__ uint8_t smem_raw[];
  return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                    ~static_cast<uintptr_t>(1023));
}

// Stages one fragment of raw accumulator values in this CTA's split-K
// staging buffer (its idle ring), float4 slot (f * 8 + j4) * kEpiThreads +
// epilogue thread: a warp writes 512 contiguous bytes.
template <int kEpiThreads>
__device__ __forceinline__ void stage_frag(float4* staging, int f, const float (&v)[32],
                                           int etid) {
#pragma unroll
  for (int j4 = 0; j4 < 8; ++j4)
    staging[(f * 8 + j4) * kEpiThreads + etid] =
        make_float4(v[4 * j4], v[4 * j4 + 1], v[4 * j4 + 2], v[4 * j4 + 3]);
}

// The cluster's CTAs are the K splits of one tile, each with its accumulator
// staged.  This CTA (rank r) takes the float4 slots r, r + NS, ... of every
// epilogue thread position, adds the NS splits' values in split order (the
// same sum whichever CTA computes it), and stores alpha * sum (+ beta C)
// with the thread position's row and column mapping.  G slots at a time, so
// that G * NS (<= 16) distributed-shared-memory loads are in flight.
template <int NS, int NF, int kEpiThreads, int EC, int BN>
__device__ __forceinline__ void cluster_split_sum_n(const TcArgs& p, const float4* staging,
                                                    int etid, int warp, int lane, int mb, int nb,
                                                    float alpha) {
  constexpr int G = 16 / NS;
  constexpr int kSlots = NF * 8;
  auto cl = cooperative_groups::this_cluster();
  const int r = static_cast<int>(cl.block_rank());
  const int row_q = mb * kBM + (warp & 3) * 32;
  const int col_s = nb * BN + ((warp - 2) / 4) * EC;
  if (row_q >= p.M || col_s >= p.N) return;
  const bool vec2 = (p.ldc % 2 == 0) && ((reinterpret_cast<uintptr_t>(p.C) & 7) == 0);
  const float4* src[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) src[s] = cl.map_shared_rank(staging, s);
#pragma unroll 1
  for (int q0 = r; q0 < kSlots; q0 += G * NS) {
    float4 c[G][NS];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int q = q0 + g * NS;
#pragma unroll
      for (int s = 0; s < NS; ++s)
        if (q < kSlots) c[g][s] = src[s][q * kEpiThreads + etid];
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int q = q0 + g * NS;
      if (q >= kSlots) break;
      float4 a = c[g][0];
#pragma unroll
      for (int s = 1; s < NS; ++s) {
        a.x += c[g][s].x;
        a.y += c[g][s].y;
        a.z += c[g][s].z;
        a.w += c[g][s].w;
      }
      const float v[4] = {a.x, a.y, a.z, a.w};
      const int f = q >> 3, j4 = q & 7;
      store_frag<1>(v, p.C, p.ldc, p.M, p.N, row_q + 16 * (f & 1),
                    col_s + 64 * (f >> 1) + 8 * j4, alpha, p.beta, vec2, lane);
    }
  }
}

// The sum above for the cluster's size (2 to 8 splits).
template <int NF, int kEpiThreads, int EC, int BN>
__device__ __forceinline__ void cluster_split_sum(const TcArgs& p, const float4* staging,
                                                  int etid, int warp, int lane, int mb, int nb,
                                                  float alpha) {
  switch (p.splits) {
#define COMPAR_SPLIT_SUM(ns)                                                                  \
  case ns:                                                                                    \
    cluster_split_sum_n<ns, NF, kEpiThreads, EC, BN>(p, staging, etid, warp, lane, mb, nb, \
                                                     alpha);                                \
    break;
    COMPAR_SPLIT_SUM(2)
    COMPAR_SPLIT_SUM(3)
    COMPAR_SPLIT_SUM(4)
    COMPAR_SPLIT_SUM(5)
    COMPAR_SPLIT_SUM(6)
    COMPAR_SPLIT_SUM(7)
    COMPAR_SPLIT_SUM(8)
#undef COMPAR_SPLIT_SUM
    default: break;
  }
}

// End of a promoted item in the epilogue: stores the tile from `sum` (a
// classic unit, or a stream-K tile with one contributor) or publishes this
// CTA's stream-K piece and takes part in the count-and-sum.  `sum` is not
// used after the store or the publication, so its registers are free for
// the sums.  False when a bounded wait gave up.
template <int NF, int kEpiThreads, int BN>
__device__ __forceinline__ bool finish_promoted(const TcArgs& p, const WorkItem& it,
                                                const float (&sum)[NF][32], uint64_t* epi_bar,
                                                uint32_t& epi_uses, volatile int* last_flag,
                                                const dev::WaitCtx& w, int etid, int lane,
                                                float* out, int64_t out_ld, int row_q, int col_s,
                                                float alpha, float beta, bool vec_out,
                                                const CUtensorMap* tmC, uint8_t* estage,
                                                uint32_t& nbox) {
  const SkPiece sp = sk_piece(p, it);
  if (p.split_cluster) {  // an in-cluster K split: the cluster adds the sums
    float4* staging = reinterpret_cast<float4*>(ring_base());
#pragma unroll
    for (int f = 0; f < NF; ++f) stage_frag<kEpiThreads>(staging, f, sum[f], etid);
    return true;
  }
  if (sp.nc == 1) {
    if (row_q < p.M && col_s < p.N) {
      if (estage != nullptr) {
#pragma unroll
        for (int f = 0; f < NF; ++f)
          tma_store_frag(tmC, estage, nbox, sum[f], row_q + 16 * (f & 1), col_s + 64 * (f >> 1),
                         p.M, p.N, alpha, lane);
      } else {
#pragma unroll
        for (int f = 0; f < NF; ++f)
          store_frag<8>(sum[f], out, out_ld, p.M, p.N, row_q + 16 * (f & 1),
                        col_s + 64 * (f >> 1), alpha, beta, vec_out, lane);
      }
    }
    return true;
  }
  float4* mine = sk_slab<BN>(p, blockIdx.x, it.piece);
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int j4 = 0; j4 < 8; ++j4)
      mine[(f * 8 + j4) * kEpiThreads + etid] =
          make_float4(sum[f][4 * j4], sum[f][4 * j4 + 1], sum[f][4 * j4 + 2], sum[f][4 * j4 + 3]);
  return sk_count_and_sum<NF, kEpiThreads, BN>(p, sp, epi_bar, epi_uses, last_flag, w, etid,
                                               lane, out, out_ld, row_q, col_s, alpha, beta,
                                               vec_out);
}

// kPair: launched in clusters of 2 CTAs (a CTA pair on one TPC).  Both CTAs
// load their halves (A rows, B rows or columns) and run the epilogue on
// their rows; the even CTA alone issues the pair's MMAs (cta_group::2).  Its
// `full` barriers count both CTAs' bytes; its commits release the stage and
// hand over the accumulator in both CTAs (multicast); both CTAs' epilogue
// warps free an accumulator on the even CTA's `tempty`.
template <int V, bool kPair>
__global__ void __launch_bounds__(Layout<V, kPair>::kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmA2,
                   const __grid_constant__ CUtensorMap tmB2,
                   const __grid_constant__ CUtensorMap tmA3,
                   const __grid_constant__ CUtensorMap tmB3,
                   const __grid_constant__ CUtensorMap tmC, const TcArgs p) {
  using T = Traits<V>;
  using L = Layout<V, kPair>;
  static_assert(!(kPair && T::fused), "the fused split runs on single CTAs only");
  constexpr int P = T::pieces;
  constexpr int BN = T::BN;
  constexpr int S = L::kStages;
  constexpr int kChunkKB = T::chunk_kb;

  uint8_t* smem = ring_base();
  uint8_t* sA = smem;                              // [S][P][kABytes]
  uint8_t* sB = smem + S * P * L::kABytes;         // [S][P][kBBytes]
  uint8_t* epi_stage = sB + S * P * L::kBBytes;   // [epi warps][2][2 KB] (TMA stores)
  uint64_t* full = reinterpret_cast<uint64_t*>(epi_stage + L::kEpiStageBytes);
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;   // [2]
  uint64_t* tempty = tfull + 2;  // [2]
  uint64_t* drain = tempty + 2;
  uint64_t* epi_bar = drain + 1;  // rendezvous of the epilogue warps (stream-K)
  uint64_t* split_done = epi_bar + 1;  // [S] fused variant: stage split, MMA may read
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(split_done + S);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* last_flag = abort_flag + 1;

  const int warp = threadIdx.x / 32;
  const int lane = threadIdx.x % 32;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      dev::mbar_init(&full[s], 1);
      dev::mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      dev::mbar_init(&tfull[a], 1);
      dev::mbar_init(&tempty[a], L::kTemptyCount);
    }
    dev::mbar_init(drain, 1);
    dev::mbar_init(epi_bar, L::kEpiThreads);
    for (int s = 0; s < S; ++s) dev::mbar_init(&split_done[s], T::epi);
    *abort_flag = 0;
    dev::fence_barrier_init();
  }
  if (warp == 0 && lane == 0) {
    dev::tma_prefetch_desc(&tmA);
    dev::tma_prefetch_desc(&tmB);
    if constexpr (P >= 2) {
      dev::tma_prefetch_desc(&tmA2);
      dev::tma_prefetch_desc(&tmB2);
    }
    if constexpr (P == 3) {
      dev::tma_prefetch_desc(&tmA3);
      dev::tma_prefetch_desc(&tmB3);
    }
    if (L::kTmaStore && p.tma_c) dev::tma_prefetch_desc(&tmC);
  }
  if (warp == 1) {
    if constexpr (kPair) {
      dev::tmem_alloc_pair(tmem_slot, L::kTmemCols);  // with the peer's warp 1
      dev::tmem_relinquish_pair();
    } else {
      dev::tmem_alloc(tmem_slot, L::kTmemCols);
      dev::tmem_relinquish();
    }
  }
  dev::tc_fence_before();
  __syncthreads();
  // a pair's barriers are all initialised before either CTA signals the other's
  if constexpr (kPair) dev::cluster_sync();
  dev::tc_fence_after();
  // launched programmatically: the set-up above overlapped the stream's
  // previous kernel (the pre-pass), whose results are read from here on
  dev::griddep_wait();
  const uint32_t tmem_base = *tmem_slot;
  const uint32_t rank = kPair ? dev::cluster_ctarank() : 0u;
  dev::WaitCtx w{abort_flag, p.err_word, p.budget_ns};
  if constexpr (kPair)
    w.peer_abort = cooperative_groups::this_cluster().map_shared_rank(
        const_cast<int*>(abort_flag), rank ^ 1u);
  // the even CTA's barriers as shared::cluster addresses (pairs only)
  const uint32_t full_lead = kPair ? dev::mapa(dev::smem_u32(full), 0) : 0u;
  const uint32_t tempty_lead = kPair ? dev::mapa(dev::smem_u32(tempty), 0) : 0u;
  // first row of this CTA's kBM rows of tile row mb
  auto tile_row0 = [&](int mb) { return (kPair ? 2 * mb + static_cast<int>(rank) : mb) * kBM; };
  WorkItem it;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer
    uint32_t stage = 0, phase = 0;
    uint32_t issued = 0, issued_parity = 0;  // per-stage bit masks
    // the even CTA's full barrier counts both CTAs' bytes of a pair's stage
    constexpr uint32_t kTx = static_cast<uint32_t>(L::kStageBytes) * (kPair ? 2 : 1);
    bool ok = true;
    for (int i = 0; ok && get_item<kChunkKB>(p, i, it); ++i) {
      int mb, nb;
      tile_coords(it.tile, p.tiles_m, p.tiles_n, mb, nb);
      const int a_row = tile_row0(mb);
      const int b_row = nb * BN + static_cast<int>(rank) * L::kBRows;  // this CTA's B half
      for (int kb = it.kb_begin; kb < it.kb_end; ++kb) {
        if (!dev::mbar_wait(&empty[stage], phase ^ 1, w)) {
          ok = false;
          break;
        }
        if (rank == 0) dev::mbar_arrive_expect_tx(&full[stage], kTx);
        auto load = [&](void* dst, const CUtensorMap* map, int cx, int cy) {
          if constexpr (kPair)
            dev::tma_load_2d_pair(dst, map, full_lead + 8u * stage, cx, cy);
          else
            dev::tma_load_2d(dst, map, &full[stage], cx, cy);
        };
        const int x = kb * L::kElemsPerStage;
        uint8_t* a_dst = sA + (stage * P) * L::kABytes;
        uint8_t* b_dst = sB + (stage * P) * L::kBBytes;
        if constexpr (T::fused) {
          // float32 tiles as stored: A [128 rows][32 K]; B box (ng, kg) =
          // [8 K][64 N] at 2048 (4 ng + kg)
          dev::tma_load_2d(a_dst, &tmA, &full[stage], x, mb * kBM);
#pragma unroll
          for (int ng = 0; ng < BN / 64; ++ng)
#pragma unroll
            for (int kg = 0; kg < 4; ++kg)
              dev::tma_load_2d(b_dst + 2048 * (4 * ng + kg), &tmB, &full[stage],
                               nb * BN + 64 * ng, x + 8 * kg);
        } else {
        load(a_dst, &tmA, x, a_row);
        if constexpr (P >= 2) load(a_dst + L::kABytes, &tmA2, x, a_row);
        if constexpr (P == 3) load(a_dst + 2 * L::kABytes, &tmA3, x, a_row);
        if constexpr (T::b_mn) {
#pragma unroll
          for (int h = 0; h < L::kBRows / 64; ++h) {
            const int n0 = b_row + h * 64;
            load(b_dst + h * L::kMnBox, &tmB, n0, x);
            if constexpr (P >= 2) load(b_dst + L::kBBytes + h * L::kMnBox, &tmB2, n0, x);
            if constexpr (P == 3) load(b_dst + 2 * L::kBBytes + h * L::kMnBox, &tmB3, n0, x);
          }
        } else {
          load(b_dst, &tmB, x, b_row);
          if constexpr (P >= 2) load(b_dst + L::kBBytes, &tmB2, x, b_row);
          if constexpr (P == 3) load(b_dst + 2 * L::kBBytes, &tmB3, x, b_row);
        }
        }
        issued |= 1u << stage;
        issued_parity = (issued_parity & ~(1u << stage)) | (phase << stage);
        if (++stage == S) {
          stage = 0;
          phase ^= 1;
        }
      }
    }
    // every load of this CTA is issued: the stream's next kernel may be
    // scheduled (it waits for this one to complete before touching memory)
    dev::griddep_launch_dependents();
    if (!ok) {
      // Let every copy this thread started land before the CTA exits (a
      // pair's copies are all counted on the even CTA's barriers).
      for (int s = 0; rank == 0 && s < S; ++s)
        if (issued & (1u << s)) drain_wait(&full[s], (issued_parity >> s) & 1, p.budget_ns);
    } else if constexpr (kPair) {
      // The even CTA's commits release this CTA's stages from afar: wait
      // until every stage filled has been released, so that no arrival is
      // still on its way when the CTA exits.
      for (int s = 0; s < S; ++s) {
        if (!dev::mbar_wait(&empty[stage], phase ^ 1, w)) break;
        if (++stage == S) {
          stage = 0;
          phase ^= 1;
        }
      }
    }
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ------------------------------------------------------------ MMA issuer
    constexpr uint32_t idesc = T::b_mn ? dev::make_idesc_bmn(T::fmt, T::fmt, L::kMmaM, BN)
                                       : dev::make_idesc(T::fmt, T::fmt, L::kMmaM, BN);
    auto mma_op = [&](uint32_t d, uint64_t a, uint64_t b, uint32_t accumulate) {
      if constexpr (kPair)
        dev::mma_pair<T::kind>(d, a, b, idesc, accumulate);
      else
        dev::mma<T::kind>(d, a, b, idesc, accumulate);
    };
    // release / hand over in this CTA, or in both CTAs of a pair
    auto commit = [&](uint64_t* bar) {
      if constexpr (kPair)
        dev::mma_commit_pair_mc(bar, 0x3);
      else
        dev::mma_commit(bar);
    };
    uint32_t stage = 0, phase = 0;
    int acc_iter = 0;  // accumulator-buffer uses (one per K chunk)
    bool ok = true;
    for (int i = 0; ok && get_item<kChunkKB>(p, i, it); ++i) {
      const int kb_begin = it.kb_begin, kb_end = it.kb_end;
      const int chunk = kChunkKB > 0 ? kChunkKB : kb_end - kb_begin;
      for (int kb0 = kb_begin; ok && kb0 < kb_end; kb0 += chunk, ++acc_iter) {
        const uint32_t acc = acc_iter & 1;
        const uint32_t acc_phase = (acc_iter >> 1) & 1;
        if (!dev::mbar_wait(&tempty[acc], acc_phase ^ 1, w)) {
          ok = false;
          break;
        }
        dev::tc_fence_after();
        const uint32_t d_tmem = tmem_base + acc * BN;
        const int kb_stop = min(kb_end, kb0 + chunk);
        for (int kb = kb0; kb < kb_stop; ++kb) {
          if (!dev::mbar_wait(T::fused ? &split_done[stage] : &full[stage], phase, w)) {
            ok = false;
            break;
          }
          dev::tc_fence_after();
          const uint32_t a0 = dev::smem_u32(sA + (stage * P) * L::kABytes);
          const uint32_t b0 = dev::smem_u32(sB + (stage * P) * L::kBBytes);
          // Descriptors of K step kk: A (K-major) advances 32 bytes inside its
          // swizzled rows; an MN-major B advances 16 K rows (2048 bytes).
          auto b_desc = [&](int piece, int kk) -> uint64_t {
            if constexpr (T::fused)  // MN-major: a K step of 16 rows is two 8-row groups
              return dev::smem_desc_sw128_mnmajor_strided(b0 + piece * 1024 + kk * 4096, 8192,
                                                          2048);
            const uint32_t base = b0 + piece * L::kBBytes;
            if constexpr (T::b_mn)
              return dev::smem_desc_sw128_mnmajor(base + kk * 2048, L::kMnBox);
            else
              return dev::smem_desc_kmajor<T::row>(base) + (static_cast<uint64_t>(kk * 32) >> 4);
          };
          auto a_desc = [&](int piece, int kk) -> uint64_t {
            if constexpr (T::fused)
              return dev::smem_desc_sw64_kmajor_strided(a0 + piece * 512, 1024) +
                     (static_cast<uint64_t>(kk * 32) >> 4);
            return dev::smem_desc_kmajor<T::row>(a0 + piece * L::kABytes) +
                   (static_cast<uint64_t>(kk * 32) >> 4);
          };
          if constexpr (P == 3) {
            // small products of every K step of the stage, then the leading ones
#pragma unroll
            for (int kk = 0; kk < T::row / 32; ++kk) {
              const uint32_t first = (kb == kb0 && kk == 0) ? 0u : 1u;
              const uint64_t a_0 = a_desc(0, kk), a_1 = a_desc(1, kk), a_2 = a_desc(2, kk);
              const uint64_t b_0 = b_desc(0, kk), b_1 = b_desc(1, kk), b_2 = b_desc(2, kk);
              mma_op(d_tmem, a_0, b_1, first);
              mma_op(d_tmem, a_1, b_0, 1u);
              mma_op(d_tmem, a_0, b_2, 1u);
              mma_op(d_tmem, a_1, b_1, 1u);
              mma_op(d_tmem, a_2, b_0, 1u);
            }
#pragma unroll
            for (int kk = 0; kk < T::row / 32; ++kk)
              mma_op(d_tmem, a_desc(0, kk), b_desc(0, kk), 1u);
          }
          if constexpr (P == 2 && T::small_first) {
            // the cross products of every K step of the stage, then hi * hi
#pragma unroll
            for (int kk = 0; kk < T::row / 32; ++kk) {
              const uint32_t first = (kb == kb0 && kk == 0) ? 0u : 1u;
              mma_op(d_tmem, a_desc(0, kk), b_desc(1, kk), first);
              mma_op(d_tmem, a_desc(1, kk), b_desc(0, kk), 1u);
            }
#pragma unroll
            for (int kk = 0; kk < T::row / 32; ++kk)
              mma_op(d_tmem, a_desc(0, kk), b_desc(0, kk), 1u);
          }
#pragma unroll
          for (int kk = 0; P < 3 && !T::small_first && kk < T::row / 32; ++kk) {
            const uint32_t first = (kb == kb0 && kk == 0) ? 0u : 1u;
            if constexpr (P == 2) {
              mma_op(d_tmem, a_desc(0, kk), b_desc(0, kk), first);
              mma_op(d_tmem, a_desc(0, kk), b_desc(1, kk), 1u);
              mma_op(d_tmem, a_desc(1, kk), b_desc(0, kk), 1u);
            } else {
              mma_op(d_tmem, a_desc(0, kk), b_desc(0, kk), first);
            }
          }
          commit(&empty[stage]);  // stage reusable once these MMAs finish
          if (++stage == S) {
            stage = 0;
            phase ^= 1;
          }
        }
        if (!ok) break;
        commit(&tfull[acc]);  // chunk accumulator ready for the epilogue
      }
    }
    // All MMAs issued by this thread complete before TMEM is released.
    if constexpr (kPair)
      dev::mma_commit_pair_mc(drain, 0x1);
    else
      dev::mma_commit(drain);
    drain_wait(drain, 0, p.budget_ns);
  } else if (warp >= 2) {
    // ------------------------------------------------------------ epilogue
    // The accumulator is read in 16-row x 64-column fragments (16x256b
    // shape): four consecutive lanes hold 8 consecutive columns of a row, so
    // every store instruction writes whole 32-byte sectors of 8 rows.
    const int quarter = warp & 3;            // TMEM lanes this warp may access
    const int cslice = (warp - 2) / 4;       // which kEpiCols-wide column slice
    constexpr int EC = L::kEpiCols;
    constexpr int NF = 2 * (EC / 64);        // fragments: 2 row halves x EC/64 column blocks
    static_assert(EC % 64 == 0, "epilogue column slice");
    float alpha = p.alpha;
    if (p.dequant_a) alpha *= *p.dequant_a;
    if (p.dequant_b) alpha *= *p.dequant_b;
    const bool vec2 = (p.ldc % 2 == 0) && ((reinterpret_cast<uintptr_t>(p.C) & 7) == 0);
    int acc_iter = 0;
    bool ok = true;
    // split units write alpha * partial (no beta) into their own slab
    const bool split = p.splits > 1;
    const int64_t out_ld = split ? p.N : p.ldc;
    const bool vec_out = split ? (p.N % 2 == 0) : vec2;
    const float beta = split ? 0.f : p.beta;
    uint32_t epi_uses = 0;  // completed phases of epi_bar
    // TMA-store epilogue: this warp's staging boxes (null: plain stores) and
    // the boxes it has staged so far
    uint32_t nbox = 0;
    auto estage = [&]() -> uint8_t* {
      return L::kTmaStore && p.tma_c ? epi_stage + (warp - 2) * L::kEpiWarpBytes : nullptr;
    };
    const int etid = threadIdx.x - 64;
    // this warp is done reading accumulator `acc`: every thread arrives, or
    // in a pair one lane per warp on the even CTA's barrier (tcgen05.ld
    // waits are warp-wide, so the warp's loads are complete)
    auto release_acc = [&](uint32_t acc) {
      dev::tc_fence_before();
      if constexpr (kPair) {
        __syncwarp();
        if (lane == 0) dev::mbar_arrive_cluster(tempty_lead + 8u * acc);
      } else {
        dev::mbar_arrive(&tempty[acc]);
      }
    };
    if constexpr (T::fused) {
      // The epilogue warps also split the stages: each stage is split as
      // soon as TMA has landed it, and a K chunk is promoted once the split
      // has run kLag stages past the chunk's end, so the MMA still has split
      // stages queued while these warps read TMEM or store a tile.
      constexpr int kLag = 2;
      const int cw = warp - 2;
      uint32_t stage = 0, phase = 0;
      int g = 0;              // stages split so far
      WorkItem cit, pit;      // split cursor, promotion cursor
      int ci = 0;
      bool c_have = get_item<kChunkKB>(p, 0, cit);
      int ckb = cit.kb_begin;
      int p_g0 = 0;           // split index of the promotion item's first stage
      for (int pi = 0; ok && get_item<kChunkKB>(p, pi, pit); ++pi) {
        // one promoted item: sum lives only here
        float sum[NF][32];
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
          for (int j = 0; j < 32; ++j) sum[f][j] = 0.f;
        for (int kb0 = pit.kb_begin; ok && kb0 < pit.kb_end; kb0 += kChunkKB) {
          // split up to kLag stages past this chunk's last stage
          const int last = p_g0 + min(pit.kb_end, kb0 + kChunkKB) - pit.kb_begin - 1;
          while (c_have && g <= last + kLag) {
            if (!dev::mbar_wait(&full[stage], phase, w)) {
              ok = false;
              break;
            }
            split_stage_in_place<T::epi>(sA + (stage * P) * L::kABytes,
                                         sB + (stage * P) * L::kBBytes, cw, lane);
            dev::fence_proxy_async_smem();  // generic writes before the MMA's reads
            __syncwarp();
            if (lane == 0) dev::mbar_arrive(&split_done[stage]);
            if (++stage == S) {
              stage = 0;
              phase ^= 1;
            }
            ++g;
            if (++ckb == cit.kb_end) {
              c_have = get_item<kChunkKB>(p, ++ci, cit);
              if (c_have) ckb = cit.kb_begin;
            }
          }
          if (!ok) break;
          const uint32_t acc = acc_iter & 1;
          const uint32_t acc_phase = (acc_iter >> 1) & 1;
          if (!dev::mbar_wait(&tfull[acc], acc_phase, w)) {
            ok = false;
            break;
          }
          dev::tc_fence_after();
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            uint32_t r[32];
            dev::tmem_ld_16x256b_x8(
                tmem_base + (static_cast<uint32_t>(quarter * 32 + 16 * (f & 1)) << 16) +
                    acc * BN + cslice * EC + 64 * (f >> 1),
                r);
            dev::tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 32; ++j) sum[f][j] += __uint_as_float(r[j]);
          }
          release_acc(acc);
          ++acc_iter;
        }
        if (!ok) break;
        int mb, nb;
        tile_coords(pit.tile, p.tiles_m, p.tiles_n, mb, nb);
        const int row_q = tile_row0(mb) + quarter * 32;
        const int col_s = nb * BN + cslice * EC;
        float* out = split ? p.partial + static_cast<int64_t>(pit.split) * p.M * p.N : p.C;
        if (!finish_promoted<NF, L::kEpiThreads, BN>(p, pit, sum, epi_bar, epi_uses, last_flag,
                                                     w, etid, lane, out, out_ld, row_q, col_s,
                                                     alpha, beta, vec_out, &tmC, estage(), nbox)) {
          ok = false;
          break;
        }
        p_g0 += pit.kb_end - pit.kb_begin;
      }
    }
    for (int i = 0; !T::fused && ok && get_item<kChunkKB>(p, i, it); ++i) {
      int mb, nb;
      tile_coords(it.tile, p.tiles_m, p.tiles_n, mb, nb);
      const int num_chunks =
          kChunkKB > 0 ? (it.kb_end - it.kb_begin + kChunkKB - 1) / kChunkKB : 1;
      float* out = split ? p.partial + static_cast<int64_t>(it.split) * p.M * p.N : p.C;
      const int row_q = tile_row0(mb) + quarter * 32;     // first row of this warp's quarter
      const int col_s = nb * BN + cslice * EC;       // first column of its slice
      auto frag_taddr = [&](uint32_t acc, int f) {
        return tmem_base + (static_cast<uint32_t>(quarter * 32 + 16 * (f & 1)) << 16) +
               acc * BN + cslice * EC + 64 * (f >> 1);
      };
      if constexpr (kChunkKB > 0) {
        // Promotion: each K chunk's TMEM partial sum is added into FP32
        // registers (round to nearest), so the tensor core's accumulator
        // only ever sums kChunkKB k-blocks.
        float sum[NF][32];
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
          for (int j = 0; j < 32; ++j) sum[f][j] = 0.f;
        for (int ch = 0; ch < num_chunks; ++ch, ++acc_iter) {
          const uint32_t acc = acc_iter & 1;
          const uint32_t acc_phase = (acc_iter >> 1) & 1;
          if (!dev::mbar_wait(&tfull[acc], acc_phase, w)) {
            ok = false;
            break;
          }
          dev::tc_fence_after();
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            uint32_t r[32];
            dev::tmem_ld_16x256b_x8(frag_taddr(acc, f), r);
            dev::tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 32; ++j) sum[f][j] += __uint_as_float(r[j]);
          }
          release_acc(acc);
        }
        if (!ok) break;
        if (!finish_promoted<NF, L::kEpiThreads, BN>(p, it, sum, epi_bar, epi_uses, last_flag, w,
                                                     etid, lane, out, out_ld, row_q, col_s,
                                                     alpha, beta, vec_out, &tmC, estage(), nbox)) {
          ok = false;
          break;
        }
        continue;
      }
      const uint32_t acc = acc_iter & 1;
      const uint32_t acc_phase = (acc_iter >> 1) & 1;
      ++acc_iter;
      if (!dev::mbar_wait(&tfull[acc], acc_phase, w)) break;
      dev::tc_fence_after();
      const SkPiece sp = sk_piece(p, it);
      if (sp.nc > 1) {
        // stream-K piece: publish the accumulator straight from TMEM, free
        // it, then count in (and sum the tile if this CTA is the last)
        float4* mine = sk_slab<BN>(p, blockIdx.x, it.piece);
#pragma unroll 1
        for (int f = 0; f < NF; ++f) {
          uint32_t r[32];
          dev::tmem_ld_16x256b_x8(frag_taddr(acc, f), r);
          dev::tmem_ld_wait();
#pragma unroll
          for (int j4 = 0; j4 < 8; ++j4)
            mine[(f * 8 + j4) * L::kEpiThreads + etid] =
                make_float4(__uint_as_float(r[4 * j4]), __uint_as_float(r[4 * j4 + 1]),
                            __uint_as_float(r[4 * j4 + 2]), __uint_as_float(r[4 * j4 + 3]));
        }
        release_acc(acc);
        if (!sk_count_and_sum<NF, L::kEpiThreads, BN>(p, sp, epi_bar, epi_uses, last_flag, w,
                                                      etid, lane, out, out_ld, row_q, col_s,
                                                      alpha, beta, vec_out))
          break;
        continue;
      }
#pragma unroll 1
      for (int f = 0; f < NF; ++f) {
        uint32_t r[32];
        dev::tmem_ld_16x256b_x8(frag_taddr(acc, f), r);
        dev::tmem_ld_wait();
        float v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
        // an in-cluster K split stages the accumulator in the ring, idle by
        // now (a CTA of a K split has one item: no copy or MMA is left)
        if (p.split_cluster)
          stage_frag<L::kEpiThreads>(reinterpret_cast<float4*>(ring_base()), f, v, etid);
        else if (L::kTmaStore && p.tma_c)
          tma_store_frag(&tmC, estage(), nbox, v, row_q + 16 * (f & 1), col_s + 64 * (f >> 1),
                         p.M, p.N, alpha, lane);
        else if (row_q < p.M && col_s < p.N)
          store_frag<8>(v, out, out_ld, p.M, p.N, row_q + 16 * (f & 1), col_s + 64 * (f >> 1),
                          alpha, beta, vec_out, lane);
      }
      release_acc(acc);
    }
  }

  // the TMA-store epilogue's last stores have read their staging boxes (and
  // are complete) before the CTA can leave
  if (L::kTmaStore && p.tma_c && warp >= 2 && lane == 0) dev::bulk_wait_all();
  __syncthreads();
  if constexpr (!kPair) {
    if (p.split_cluster) {
      // every CTA of the cluster has staged its split (or given up: the sum
      // is then wrong, and the error word says so)
      dev::cluster_sync();
      if (warp >= 2 && get_item<kChunkKB>(p, 0, it)) {
        int mb, nb;
        tile_coords(it.tile, p.tiles_m, p.tiles_n, mb, nb);
        float alpha = p.alpha;
        if (p.dequant_a) alpha *= *p.dequant_a;
        if (p.dequant_b) alpha *= *p.dequant_b;
        constexpr int EC = L::kEpiCols;
        cluster_split_sum<2 * (EC / 64), L::kEpiThreads, EC, BN>(
            p, reinterpret_cast<const float4*>(sA), static_cast<int>(threadIdx.x) - 64, warp,
            lane, mb, nb, alpha);
      }
      dev::cluster_sync();  // no CTA leaves while a peer still reads its staging
    }
  }
  // a pair frees its tensor memory together, once both CTAs are done (the
  // even CTA has drained every MMA writing into the odd CTA's columns)
  if constexpr (kPair) dev::cluster_sync();
  if (warp == 1) {
    dev::tc_fence_after();
    if constexpr (kPair)
      dev::tmem_dealloc_pair(tmem_base, L::kTmemCols);
    else
      dev::tmem_dealloc(tmem_base, L::kTmemCols);
  }
}

// ------------------------------------------------------------------ timeout self-test
__global__ void timeout_selftest_kernel(int* err_word, unsigned long long budget_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    dev::mbar_init(&bar, 1);
    abort_flag = 0;
    dev::fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const dev::WaitCtx w{&abort_flag, err_word, budget_ns};
    // Nothing ever arrives on `bar`: the bounded wait runs out and records
    // the timeout status, then the kernel returns.
    (void)dev::mbar_wait(&bar, 0, w);
  }
}

// ------------------------------------------------------------------ host side
int round_up(int64_t x, int64_t m) { return static_cast<int>((x + m - 1) / m * m); }

CUtensorMapDataType map_type(int v) {
  switch (v) {
    case COMPAR_V_TC_TF32:
    case COMPAR_V_SPLIT3_TF32:
    case COMPAR_V_SPLIT3_FUSED: return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    case COMPAR_V_TC_FP8: return CU_TENSOR_MAP_DATA_TYPE_UINT8;
    default: return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  }
}

// Launch plan of a tensor-core call: K blocks, tiles, and the split of K
// when the tiles alone would leave most SMs idle (at least 8 K blocks per
// split, at most one unit per SM).  A partial last wave of tiles is cut
// into stream-K pieces instead (whole chunks: the promotion chunk, or
// kPlainSkChunk K blocks for the variants without promotion; at least a
// quarter tile each, so that a tile has at most five contributors), when
// that shortens the wave by a quarter or more and saves more time than the
// fixup costs.
struct TcPlan {
  int num_kb, tiles, splits, kb_per;
  int sk_tile0 = 0, sk_cpt = 0, sk_q = 0, sk_ctas = 0;
};

// Tile width of every tensor-core variant (stream-K piece size on the host).
constexpr int kTileN = 256;
static_assert(Traits<COMPAR_V_TC_TF32>::BN == kTileN && Traits<COMPAR_V_TC_BF16>::BN == kTileN &&
                  Traits<COMPAR_V_TC_FP8>::BN == kTileN && Traits<COMPAR_V_SPLIT3>::BN == kTileN &&
                  Traits<COMPAR_V_SPLIT6>::BN == kTileN &&
                  Traits<COMPAR_V_SPLIT3_TF32>::BN == kTileN &&
                  Traits<COMPAR_V_SPLIT3_FUSED>::BN == kTileN,
              "stream-K pieces are kBM x kTileN");

// K blocks per stream-K chunk: the promotion chunk where there is one.
int sk_chunk_of(int v) {
  switch (v) {
    case COMPAR_V_SPLIT3: return Traits<COMPAR_V_SPLIT3>::chunk_kb;
    case COMPAR_V_SPLIT6: return Traits<COMPAR_V_SPLIT6>::chunk_kb;
    case COMPAR_V_SPLIT3_TF32: return Traits<COMPAR_V_SPLIT3_TF32>::chunk_kb;
    case COMPAR_V_SPLIT3_FUSED: return Traits<COMPAR_V_SPLIT3_FUSED>::chunk_kb;
    default: return kPlainSkChunk;
  }
}

// Time of one 128 x 256 tile's MMAs over K (us) at the sustained per-SM
// tensor rate of the variant's kind (bf16 ~9.4e12 flop/s per SM; fp8 twice,
// tf32 half), times its products per output.
double tile_us(int v, int64_t k) {
  double rate = 9.4e12, products = 1;
  switch (v) {
    case COMPAR_V_TC_FP8: rate *= 2; break;
    case COMPAR_V_TC_TF32: rate /= 2; break;
    case COMPAR_V_SPLIT3:
    case COMPAR_V_SPLIT3_FUSED: products = 3; break;
    case COMPAR_V_SPLIT6: products = 6; break;
    case COMPAR_V_SPLIT3_TF32: rate /= 2; products = 3; break;
    default: break;
  }
  return 2.0 * kBM * kTileN * static_cast<double>(k) * products / rate * 1e6;
}

// The stream-K fixup (publish a 128 KB piece, count, the last contributor
// sums 2-5 of them) costs ~10 us; a tail cut is taken only when it saves
// clearly more.
constexpr double kSkMinSavingUs = 12.0;

// `slots`: SMs, or CTA pairs that can run at once when `pair` (tiles are
// then 2 kBM x 256 and K is never split: pairs serve calls with a wave of
// tiles or more).
TcPlan tc_plan(int v, const GemmCall& c, int slots, bool pair = false) {
  const int num_sms = slots;
  const int kelems = v == COMPAR_V_TC_FP8 ? 128
                     : v == COMPAR_V_TC_BF16 ? 64
                     : v == COMPAR_V_SPLIT3_TF32 ? 16
                                                 : 32;
  const int tile_m = pair ? 2 * kBM : kBM;
  TcPlan p;
  p.num_kb = static_cast<int>((c.k + kelems - 1) / kelems);
  p.tiles = static_cast<int>(((c.m + tile_m - 1) / tile_m) * ((c.n + 255) / 256));
  p.splits = 1;
  p.kb_per = p.num_kb;
  if (!pair && p.tiles * 2 <= num_sms && p.num_kb >= 16) {
    const int sp = std::min(num_sms / p.tiles, p.num_kb / 8);
    if (sp > 1) {
      p.kb_per = (p.num_kb + sp - 1) / sp;
      p.splits = (p.num_kb + p.kb_per - 1) / p.kb_per;
    }
  }
  const int chunk = sk_chunk_of(v);
  const int rem = p.tiles % num_sms;
  if (chunk > 0 && p.splits == 1 && rem > 0) {
    const int64_t cpt = (p.num_kb + chunk - 1) / chunk;
    const int64_t q = static_cast<int64_t>(rem) * cpt;
    const int64_t lmin = std::max<int64_t>(1, (cpt + 3) / 4);
    const int64_t ctas = std::min<int64_t>(num_sms, q / lmin);
    // worth it only when the tail wave shrinks by a quarter or more and the
    // time saved clearly exceeds the fixup's
    const int64_t longest = ctas >= 1 ? (q + ctas - 1) / ctas : cpt;
    const double saved_us = tile_us(v, c.k) * (1.0 - static_cast<double>(longest) / cpt);
    if (cpt >= 2 && ctas >= 1 && q < (int64_t{1} << 30) && 4 * longest <= 3 * cpt &&
        saved_us >= kSkMinSavingUs) {
      p.sk_tile0 = p.tiles - rem;
      p.sk_cpt = static_cast<int>(cpt);
      p.sk_q = static_cast<int>(q);
      p.sk_ctas = static_cast<int>(ctas);
    }
  }
  return p;
}

// Launch configuration of the kernel: clusters of 2 for CTA pairs, of
// `cluster` CTAs for an in-cluster K split; `programmatic`: the kernel may
// start (and run its set-up) before the stream's previous kernel completes.
// attr: room for two attributes.
template <int V, bool kPair>
cudaLaunchConfig_t tc_launch_config(int grid, cudaStream_t s, cudaLaunchAttribute* attr,
                                    int cluster = 1, bool programmatic = false) {
  using L = Layout<V, kPair>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(L::kThreads);
  cfg.dynamicSmemBytes = L::kSmemBytes;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 0;
  if (kPair || cluster > 1) {
    attr[cfg.numAttrs].id = cudaLaunchAttributeClusterDimension;
    attr[cfg.numAttrs].val.clusterDim.x = kPair ? 2 : cluster;
    attr[cfg.numAttrs].val.clusterDim.y = 1;
    attr[cfg.numAttrs].val.clusterDim.z = 1;
    ++cfg.numAttrs;
  }
  if (programmatic) {
    attr[cfg.numAttrs].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[cfg.numAttrs].val.programmaticStreamSerializationAllowed = 1;
    ++cfg.numAttrs;
  }
  return cfg;
}

// Largest in-cluster K split (portable cluster size).
constexpr int kMaxSplitCluster = 8;

// Clusters of `cs` single CTAs of variant V that can be resident at once on
// the current device (queried once per device and size; 0 when the query
// fails or there is no usable device).
template <int V>
int tc_split_cluster_capacity(int cs) {
  static std::once_flag once[kMaxDevices][kMaxSplitCluster + 1];
  static int cap[kMaxDevices][kMaxSplitCluster + 1] = {};
  if (cs < 2 || cs > kMaxSplitCluster) return 0;
  const int d = current_device_index();
  if (d < 0) return 0;
  std::call_once(once[d][cs], [d, cs] {
    cudaLaunchAttribute attr[2];
    cudaLaunchConfig_t cfg = tc_launch_config<V, false>(cs, nullptr, attr, cs);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, tc_gemm_kernel<V, false>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      n = 0;
    }
    cap[d][cs] = n;
  });
  return cap[d][cs];
}

// Shared-memory opt-in of the kernel, once per device; for pairs also the
// number of pairs that can be resident at once (pairs need two SMs of one
// TPC, so it can be below half the SM count).
template <int V, bool kPair>
int tc_kernel_setup(int* pairs_out) {
  using L = Layout<V, kPair>;
  static std::once_flag once[kMaxDevices];
  static cudaError_t err[kMaxDevices] = {};
  static int pairs[kMaxDevices] = {};
  const int d = current_device_index();
  if (d < 0) {
    set_last_error_text("tensor-core kernel set-up: no usable current device");
    return COMPAR_ERR_CUDA;
  }
  std::call_once(once[d], [d] {
    err[d] = cudaFuncSetAttribute(tc_gemm_kernel<V, kPair>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, L::kSmemBytes);
    if (err[d] == cudaSuccess && kPair) {
      cudaLaunchAttribute attr[2];
      cudaLaunchConfig_t cfg = tc_launch_config<V, kPair>(2, nullptr, attr);
      err[d] = cudaOccupancyMaxActiveClusters(&pairs[d], tc_gemm_kernel<V, kPair>, &cfg);
      if (err[d] == cudaSuccess && pairs[d] < 1) err[d] = cudaErrorInvalidConfiguration;
    }
  });
  if (err[d] != cudaSuccess) {
    set_last_cuda_error(err[d], "tensor-core kernel set-up", __FILE__, __LINE__);
    return COMPAR_ERR_CUDA;
  }
  if (pairs_out) *pairs_out = pairs[d];
  return COMPAR_OK;
}

template <int V, bool kPair>
int run_tc(const GemmCall& c, const void* A, int64_t lda, const void* B, int64_t ldb,
           const void* A2, const void* B2, const void* A3, const void* B3, const float* dq_a,
           const float* dq_b, const TcPlan& plan, float* partial, float* sk_slab,
           unsigned long long* sk_count, unsigned int sk_epoch, const DeviceGuard& g, int slots,
           cudaStream_t s) {
  using L = Layout<V, kPair>;
  using T = Traits<V>;
  int rc0 = tc_kernel_setup<V, kPair>(nullptr);
  if (rc0 != COMPAR_OK) return rc0;
  if (kPair && plan.splits > 1) return COMPAR_ERR_INVALID;
  CUtensorMap ta, tb, ta2, tb2, ta3, tb3;
  const CUtensorMapDataType dt = map_type(V);
  const uint32_t box_k = static_cast<uint32_t>(L::kElemsPerStage);
  // A: M rows of K.  B: N rows of K (K-major), or, MN-major, K rows of N
  // read in 64-column boxes.
  auto enc_b = [&](CUtensorMap* m, const void* base) {
    if constexpr (T::b_mn)
      return tma_encode_2d(m, dt, 2, base, c.n, c.k, ldb, 64, box_k, 128);
    else
      return tma_encode_2d(m, dt, T::elem, base, c.k, c.n, ldb, box_k, L::kBRows, T::row);
  };
  int rc;
  if constexpr (T::fused) {
    // float32 A [rows][K] in boxes of 32 K x 128 rows, B [K][N] in boxes of
    // 64 N x 8 K, unswizzled (the kernel splits them in shared memory)
    rc = tma_encode_2d(&ta, dt, 4, A, c.k, c.m, lda, box_k, kBM, 0);
    if (rc == COMPAR_OK) rc = tma_encode_2d(&tb, dt, 4, B, c.n, c.k, ldb, 64, 8, 0);
  } else {
    rc = tma_encode_2d(&ta, dt, T::elem, A, c.k, c.m, lda, box_k, kBM, T::row);
    if (rc == COMPAR_OK) rc = enc_b(&tb, B);
  }
  if (rc != COMPAR_OK) return rc;
  ta2 = ta3 = ta;
  tb2 = tb3 = tb;
  if (T::pieces >= 2 && !T::fused) {
    rc = tma_encode_2d(&ta2, dt, T::elem, A2, c.k, c.m, lda, box_k, kBM, T::row);
    if (rc == COMPAR_OK) rc = enc_b(&tb2, B2);
    if (rc != COMPAR_OK) return rc;
  }
  if (T::pieces == 3) {
    rc = tma_encode_2d(&ta3, dt, T::elem, A3, c.k, c.m, lda, box_k, kBM, T::row);
    if (rc == COMPAR_OK) rc = enc_b(&tb3, B3);
    if (rc != COMPAR_OK) return rc;
  }
  TcArgs a{};
  a.M = static_cast<int>(c.m);
  a.N = static_cast<int>(c.n);
  a.K = static_cast<int>(c.k);
  a.num_kb = static_cast<int>((c.k + L::kElemsPerStage - 1) / L::kElemsPerStage);
  a.splits = plan.splits;
  a.kb_per_split = plan.splits > 1 ? plan.kb_per : a.num_kb;
  a.partial = partial;
  a.sk_tile0 = plan.sk_tile0;
  a.sk_cpt = plan.sk_cpt;
  a.sk_q = plan.sk_q;
  a.sk_ctas = plan.sk_ctas;
  a.sk_slab = sk_slab;
  a.sk_count = sk_count;
  a.sk_epoch = sk_epoch;
  a.pair = kPair ? 2 : 1;
  a.tiles_m = static_cast<int>((c.m + a.pair * kBM - 1) / (a.pair * kBM));
  a.tiles_n = static_cast<int>((c.n + T::BN - 1) / T::BN);
  a.alpha = c.alpha * (V == COMPAR_V_TC_FP8 ? c.scale_a * c.scale_b : 1.f);
  a.beta = c.beta;
  a.dequant_a = dq_a;
  a.dequant_b = dq_b;
  a.C = c.C;
  a.ldc = c.ldc;
  a.err_word = g.err_word;
  a.budget_ns = g.budget_ns;
  // `slots` work-list CTAs (pairs when kPair) run at once
  const int units = a.tiles_m * a.tiles_n * a.splits;
  int grid = std::min(units, slots);
  a.dp_units = units;
  if (plan.sk_q > 0) {
    // whole waves of tiles, then the stream-K tail on sk_ctas CTAs (pairs)
    if (sk_count == nullptr || sk_slab == nullptr) return COMPAR_ERR_INVALID;
    a.dp_units = plan.sk_tile0;
    grid = plan.sk_tile0 > 0 ? slots : plan.sk_ctas;
  }
  // K splits of a tile as one cluster when every cluster of the call can be
  // resident at once (one unit per CTA); otherwise partials and a reduce
  int cluster = 1;
  if constexpr (!kPair) {
    if (a.splits > 1 && a.splits <= kMaxSplitCluster && plan.sk_q == 0 && units <= slots &&
        tc_split_cluster_capacity<V>(a.splits) * a.splits >= units) {
      cluster = a.splits;
      a.split_cluster = 1;
    }
  }
  cudaLaunchAttribute attr[2];
  const cudaLaunchConfig_t cfg =
      tc_launch_config<V, kPair>(grid * a.pair, s, attr, cluster, /*programmatic=*/true);
  cudaEvent_t ev = g.prof ? g.prof->begin(s) : nullptr;
  // C through the TMA-store epilogue where it applies (otherwise tc is an
  // unused copy of ta).  Rows of C must be whole 16-byte chunks (N a
  // multiple of 4): a bulk-tensor store clipped at the row's end was measured
  // writing the rest of the last 16-byte chunk, i.e. columns N .. N rounded
  // up to 4, which with ldc > N are the caller's.
  CUtensorMap tc = ta;
  if (L::kTmaStore && c.beta == 0.f && a.splits == 1 && c.n % 4 == 0 &&
      tma_encode_2d(&tc, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, c.C, c.n, c.m, c.ldc, 32, 16, 128) ==
          COMPAR_OK)
    a.tma_c = 1;
  COMPAR_CUDA_TRY(cudaLaunchKernelEx(&cfg, tc_gemm_kernel<V, kPair>, ta, tb, ta2, tb2, ta3, tb3,
                                     tc, a));
  if (g.prof) g.prof->end(ev, s, V);
  count_launch();
  // the split units already applied alpha (and the dequantisation)
  if (a.splits > 1 && !a.split_cluster)
    return launch_splitk_reduce(a.M, a.N, a.splits, partial, 1.f, c.beta, c.C, c.ldc, slots, s);
  return COMPAR_OK;
}

bool tma_operand_ok(const void* p, int64_t ld, int elem) {
  return (reinterpret_cast<uintptr_t>(p) % 16 == 0) && ((ld * elem) % 16 == 0);
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

bool tc_supported(int v, const GemmCall& c) {
  if (c.m > (1 << 30) || c.n > (1 << 30) || c.k > (1 << 30)) return false;
  switch (v) {
    case COMPAR_V_TC_TF32: return c.dtype == COMPAR_F32;
    case COMPAR_V_TC_BF16: return c.dtype == COMPAR_F32 || c.dtype == COMPAR_BF16;
    case COMPAR_V_TC_FP8: return c.dtype == COMPAR_F32 || c.dtype == COMPAR_F8E4M3;
    case COMPAR_V_SPLIT3:
    case COMPAR_V_SPLIT6:
    case COMPAR_V_SPLIT3_TF32: return c.dtype == COMPAR_F32;
    case COMPAR_V_SPLIT3_FUSED:
      // TMA reads the caller's float32 A and B: 16-byte rows and bases
      // (null pointers: a query about contiguous operands)
      return c.dtype == COMPAR_F32 && c.lda % 4 == 0 && c.ldb % 4 == 0 &&
             (reinterpret_cast<uintptr_t>(c.A) & 15) == 0 &&
             (reinterpret_cast<uintptr_t>(c.B) & 15) == 0;
    default: return false;
  }
}

// Whether a call runs on CTA pairs: the context's setting (-1 automatic, 0
// never, 1 whenever the variant has a pair kernel), and automatically when
// the single-CTA plan has a full wave of tiles or more.  Measured on B300
// (steady load, power-capped): pairs gain 3-4 % for 3xBF16 and 5-11 % for
// BF16 from 3072^2 up, and lose a few per cent on a single partial wave
// (2048^2).  Only the variants that hand an accumulator to the epilogue
// rarely have pair kernels; per-stage promotion (6-product split, 3xTF32)
// would put a cross-CTA handshake on every stage and measured slower.
// `pairs`: pairs resident at once.
bool has_pair_kernel(int v) {
  return v == COMPAR_V_TC_TF32 || v == COMPAR_V_TC_BF16 || v == COMPAR_V_TC_FP8 ||
         v == COMPAR_V_SPLIT3;
}

bool use_pairs(int v, const GemmCall& c, const DeviceGuard& g, int num_sms, int* pairs) {
  if (g.tc_pair == 0 || !has_pair_kernel(v)) return false;
  if (g.tc_pair < 0 && tc_plan(v, c, num_sms).tiles < num_sms) return false;
  int rc = COMPAR_ERR_INVALID;
  switch (v) {
    case COMPAR_V_TC_TF32: rc = tc_kernel_setup<COMPAR_V_TC_TF32, true>(pairs); break;
    case COMPAR_V_TC_BF16: rc = tc_kernel_setup<COMPAR_V_TC_BF16, true>(pairs); break;
    case COMPAR_V_TC_FP8: rc = tc_kernel_setup<COMPAR_V_TC_FP8, true>(pairs); break;
    case COMPAR_V_SPLIT3: rc = tc_kernel_setup<COMPAR_V_SPLIT3, true>(pairs); break;
    default: break;
  }
  return rc == COMPAR_OK && *pairs >= 1;
}

// Pre-passes + launch.  The BF16 variant reads B MN-major, K x N as stored:
// bf16 B with 16-byte rows is used in place, else converted row by row
// (pitch N rounded up to 8).  TF32, FP8 and the splits read a K-major
// (N x K) copy of B.  A is used in place when its dtype
// matches and TMA can address it, else converted.
int launch_tc(int v, const GemmCall& c, Workspace& ws, const DeviceGuard& g, int num_sms,
              cudaStream_t s) {
  if (!tc_supported(v, c)) return COMPAR_ERR_UNSUPPORTED;
  if (!tma_available()) return COMPAR_ERR_UNSUPPORTED;
  if (v == COMPAR_V_SPLIT3_FUSED) {
    // no pre-pass: workspace only for split-K partials or stream-K pieces
    const TcPlan plan = tc_plan(v, c, num_sms);
    const size_t part_bytes =
        plan.splits > 1 ? align_up(static_cast<size_t>(plan.splits) * c.m * c.n * 4, 256) : 0;
    const size_t slab_bytes =
        plan.sk_q > 0 ? static_cast<size_t>(plan.sk_ctas) * 2 * kBM * kTileN * 4 : 0;
    float* partial = nullptr;
    float* sk_slab = nullptr;
    if (part_bytes + slab_bytes > 0) {
      const int rc = ws.ensure(part_bytes + slab_bytes, s);
      if (rc != COMPAR_OK) return rc;
      uint8_t* base = static_cast<uint8_t*>(ws.ptr);
      if (part_bytes) partial = reinterpret_cast<float*>(base);
      if (slab_bytes) sk_slab = reinterpret_cast<float*>(base + part_bytes);
    }
    unsigned long long* sk_count = nullptr;
    unsigned int sk_epoch = 0;
    if (plan.sk_q > 0) {
      const int rc = ws.take_counters(static_cast<size_t>(plan.tiles), s, &sk_epoch);
      if (rc != COMPAR_OK) return rc;
      sk_count = ws.counters;
    }
    return run_tc<COMPAR_V_SPLIT3_FUSED, false>(c, c.A, c.lda, c.B, c.ldb, nullptr, nullptr, nullptr,
                                         nullptr, nullptr, nullptr, plan, partial, sk_slab,
                                         sk_count, sk_epoch, g, num_sms, s);
  }
  const int elem = (v == COMPAR_V_TC_TF32 || v == COMPAR_V_SPLIT3_TF32) ? 4
                   : (v == COMPAR_V_TC_FP8 ? 1 : 2);
  const int pieces =
      (v == COMPAR_V_SPLIT3 || v == COMPAR_V_SPLIT3_TF32) ? 2 : (v == COMPAR_V_SPLIT6 ? 3 : 1);
  const int64_t ldk = round_up(c.k, 16);  // 16-element pitch: 16-byte rows for every type
  const bool a_native = (c.dtype != COMPAR_F32 || v == COMPAR_V_TC_TF32);
  const bool a_in_place = a_native && tma_operand_ok(c.A, c.lda, elem);
  const bool fp8_from_f32 = (v == COMPAR_V_TC_FP8 && c.dtype == COMPAR_F32);
  // (MN-major B measured slower for the split variants' 64-byte stages)
  const bool b_mn = (v == COMPAR_V_TC_BF16 || v == COMPAR_V_SPLIT3);
  const int64_t ldn = round_up(c.n, 8);  // MN-major copies: 16-byte rows
  const bool b_in_place = b_mn && c.dtype == COMPAR_BF16 && tma_operand_ok(c.B, c.ldb, 2);

  // CTA pairs (cta_group::2) when the call has a wave of tiles or more
  int pairs = 0;
  const bool pair = use_pairs(v, c, g, num_sms, &pairs);
  const TcPlan plan = pair ? tc_plan(v, c, pairs, true) : tc_plan(v, c, num_sms);
  const int npair = pair ? 2 : 1;
  const size_t part_bytes =
      plan.splits > 1 ? align_up(static_cast<size_t>(plan.splits) * c.m * c.n * 4, 256) : 0;
  // stream-K: two published pieces per CTA and one counter per tail tile
  // (per CTA of a pair)
  const size_t slab_bytes =
      plan.sk_q > 0 ? static_cast<size_t>(plan.sk_ctas) * npair * 2 * kBM * kTileN * 4 : 0;
  // workspace carve: [B pieces][A pieces][fp8 scalars][split-K partials]
  const size_t a_bytes = align_up(static_cast<size_t>(c.m) * ldk * elem, 256);
  const size_t b_bytes = b_in_place ? 0
                         : b_mn     ? align_up(static_cast<size_t>(c.k) * ldn * 2, 256)
                                    : align_up(static_cast<size_t>(c.n) * ldk * elem, 256);
  // scalars: the fp8 scales (16 bytes), then the amax pass's per-block maxima
  constexpr int kMaxAmaxBlocks = 2048;
  constexpr size_t kScalBytes = 256 + 2 * kMaxAmaxBlocks * sizeof(float);
  size_t need = pieces * b_bytes + (a_in_place ? 0 : pieces * a_bytes) + kScalBytes + part_bytes +
                slab_bytes;
  int rc = ws.ensure(need, s);
  if (rc != COMPAR_OK) return rc;
  // stream-K arrival words (one per tail tile and CTA of a pair)
  unsigned long long* sk_count = nullptr;
  unsigned int sk_epoch = 0;
  if (plan.sk_q > 0) {
    rc = ws.take_counters(static_cast<size_t>(plan.tiles) * npair, s, &sk_epoch);
    if (rc != COMPAR_OK) return rc;
    sk_count = ws.counters;
  }
  uint8_t* base = static_cast<uint8_t*>(ws.ptr);
  uint8_t* wb = base;
  uint8_t* wa = base + pieces * b_bytes;
  uint8_t* scal = wa + (a_in_place ? 0 : pieces * a_bytes);
  float* fscal = reinterpret_cast<float*>(scal);              // sA, dA, sB, dB
  float* block_max = reinterpret_cast<float*>(scal + 256);    // [2 kMaxAmaxBlocks]
  float* partial = part_bytes ? reinterpret_cast<float*>(scal + kScalBytes) : nullptr;
  float* sk_slab = slab_bytes ? reinterpret_cast<float*>(scal + kScalBytes + part_bytes) : nullptr;

  int out_kind;
  switch (v) {
    case COMPAR_V_TC_TF32: out_kind = PP_COPY; break;
    case COMPAR_V_TC_BF16: out_kind = (c.dtype == COMPAR_F32) ? PP_BF16 : PP_COPY; break;
    case COMPAR_V_TC_FP8: out_kind = fp8_from_f32 ? PP_E4M3 : PP_COPY; break;
    case COMPAR_V_SPLIT3: out_kind = PP_SPLIT_BF16; break;
    case COMPAR_V_SPLIT3_TF32: out_kind = PP_SPLIT_TF32; break;
    default: out_kind = PP_SPLIT_BF16_3P; break;
  }
  const float* sa = nullptr;
  const float* sb = nullptr;
  const float* dqa = nullptr;
  const float* dqb = nullptr;
  if (fp8_from_f32) {
    int nblocks = 0;
    rc = prepass_amax2(static_cast<const float*>(c.A), c.m, c.k, c.lda,
                       static_cast<const float*>(c.B), c.k, c.n, c.ldb, block_max, kMaxAmaxBlocks,
                       num_sms, &nblocks, s);
    if (rc == COMPAR_OK) rc = prepass_fp8_scales(block_max, nblocks, fscal, s);
    if (rc != COMPAR_OK) return rc;
    sa = fscal + 0;
    dqa = fscal + 1;
    sb = fscal + 2;
    dqb = fscal + 3;
  }
  const void* Bop = wb;
  int64_t ldb_op = b_mn ? ldn : ldk;
  // float32 A and MN-major B converted row by row: one launch for both
  // when the row kernel takes them
  bool converted = false;
  if (!b_in_place && !a_in_place && b_mn && c.dtype == COMPAR_F32 && sa == nullptr) {
    const RowConvert jb{static_cast<const float*>(c.B), c.k, c.n, c.ldb, wb,
                        pieces >= 2 ? wb + b_bytes : nullptr, ldb_op, nullptr};
    const RowConvert ja{static_cast<const float*>(c.A), c.m, c.k, c.lda, wa,
                        pieces >= 2 ? wa + a_bytes : nullptr, ldk, nullptr};
    rc = prepass_convert_rows2(jb, ja, out_kind, num_sms, s);
    if (rc != COMPAR_OK && rc != COMPAR_ERR_UNSUPPORTED) return rc;
    converted = rc == COMPAR_OK;
  }
  if (b_in_place) {
    Bop = c.B;
    ldb_op = c.ldb;
  } else if (!converted) {
    // B: K x N row-major -> K x N pieces (MN-major) or N x K (K-major)
    rc = prepass_convert(c.B, c.dtype, c.k, c.n, c.ldb, wb, out_kind, ldb_op, !b_mn,
                         pieces >= 2 ? wb + b_bytes : nullptr, sb, num_sms, s);
    if (rc != COMPAR_OK) return rc;
  }
  const void* A = c.A;
  int64_t lda = c.lda;
  if (!a_in_place) {
    if (!converted) {
      rc = prepass_convert(c.A, c.dtype, c.m, c.k, c.lda, wa, out_kind, ldk, false,
                           pieces >= 2 ? wa + a_bytes : nullptr, sa, num_sms, s);
      if (rc != COMPAR_OK) return rc;
    }
    A = wa;
    lda = ldk;
  }
  const void* A2 = pieces >= 2 ? static_cast<const void*>(wa + a_bytes) : nullptr;
  const void* B2 = pieces >= 2 ? static_cast<const void*>(wb + b_bytes) : nullptr;
  const void* A3 = pieces == 3 ? static_cast<const void*>(wa + 2 * a_bytes) : nullptr;
  const void* B3 = pieces == 3 ? static_cast<const void*>(wb + 2 * b_bytes) : nullptr;
  auto run = [&](auto vtag, const float* qa, const float* qb) {
    constexpr int VV = decltype(vtag)::value;
    if constexpr (VV == COMPAR_V_TC_TF32 || VV == COMPAR_V_TC_BF16 || VV == COMPAR_V_TC_FP8 ||
                  VV == COMPAR_V_SPLIT3) {
      if (pair)
        return run_tc<VV, true>(c, A, lda, Bop, ldb_op, A2, B2, A3, B3, qa, qb, plan, partial,
                                sk_slab, sk_count, sk_epoch, g, pairs, s);
    }
    return run_tc<VV, false>(c, A, lda, Bop, ldb_op, A2, B2, A3, B3, qa, qb, plan, partial,
                             sk_slab, sk_count, sk_epoch, g, num_sms, s);
  };
  switch (v) {
    case COMPAR_V_TC_TF32:
      return run(std::integral_constant<int, COMPAR_V_TC_TF32>{}, nullptr, nullptr);
    case COMPAR_V_TC_BF16:
      return run(std::integral_constant<int, COMPAR_V_TC_BF16>{}, nullptr, nullptr);
    case COMPAR_V_TC_FP8:
      return run(std::integral_constant<int, COMPAR_V_TC_FP8>{}, dqa, dqb);
    case COMPAR_V_SPLIT3:
      return run(std::integral_constant<int, COMPAR_V_SPLIT3>{}, nullptr, nullptr);
    case COMPAR_V_SPLIT3_TF32:
      return run(std::integral_constant<int, COMPAR_V_SPLIT3_TF32>{}, nullptr, nullptr);
    default:
      return run(std::integral_constant<int, COMPAR_V_SPLIT6>{}, nullptr, nullptr);
  }
}

int tc_plan_info(int v, int64_t m, int64_t n, int64_t k, int slots, int64_t* out, bool pair) {
  if (v < COMPAR_V_TC_TF32 || v >= COMPAR_V_COUNT || v == COMPAR_V_GROUPED || m < 1 || n < 1 ||
      k < 1 || slots < 1 || !out || m > (1 << 30) || n > (1 << 30) || k > (1 << 30) ||
      (pair && !has_pair_kernel(v)))
    return COMPAR_ERR_INVALID;
  GemmCall c;
  c.m = m;
  c.n = n;
  c.k = k;
  const TcPlan p = tc_plan(v, c, slots, pair);
  const int64_t vals[9] = {p.num_kb, p.tiles,   p.splits, p.kb_per,      p.sk_tile0,
                           p.sk_cpt, p.sk_q,    p.sk_ctas, sk_chunk_of(v)};
  for (int i = 0; i < 9; ++i) out[i] = vals[i];
  return COMPAR_OK;
}

int launch_timeout_selftest(const DeviceGuard& g, cudaStream_t s) {
  timeout_selftest_kernel<<<1, 32, 0, s>>>(g.err_word, g.budget_ns);
  COMPAR_CUDA_TRY(cudaGetLastError());
  count_launch();
  return COMPAR_OK;
}

}  // namespace compar
