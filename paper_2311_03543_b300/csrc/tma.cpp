// TMA tensor-map encoding.  cuTensorMapEncodeTiled is a driver API call; it
// is resolved at run time through the runtime's driver entry-point query so
// the library does not link libcuda directly.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <unordered_map>

#include "common.h"

namespace compar {
namespace {

// Encoded maps are cached by their full argument list: a tensor map depends
// on nothing else, so a hit is exactly the map the driver would return.
// Batched calls encode hundreds of maps per call; with the cache a repeated
// batch encodes none.
struct MapKey {
  uintptr_t base;
  uint64_t inner, outer, ld;
  uint32_t box_inner, box_outer;
  int dt, elem, swizzle;
  bool operator==(const MapKey& o) const { return memcmp(this, &o, sizeof(MapKey)) == 0; }
};
struct MapKeyHash {
  size_t operator()(const MapKey& k) const {
    const auto* p = reinterpret_cast<const unsigned char*>(&k);
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < sizeof(MapKey); ++i) {
      h ^= p[i];
      h *= 1099511628211ull;
    }
    return static_cast<size_t>(h);
  }
};
constexpr size_t kMapCacheMax = 1 << 16;
std::mutex g_cache_mu;
std::unordered_map<MapKey, CUtensorMap, MapKeyHash>* g_cache = nullptr;

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn g_encode = nullptr;
std::once_flag g_once;

void resolve() {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    g_encode = reinterpret_cast<EncodeFn>(fn);
  else
    (void)cudaGetLastError();
}

}  // namespace

bool tma_available() {
  std::call_once(g_once, resolve);
  return g_encode != nullptr;
}

// 2-D map over a row-major matrix: `inner` contiguous elements per row,
// `outer` rows, row pitch `ld_elems`.  Box = box_inner x box_outer elements
// whose rows are exactly one swizzle width (64 or 128 bytes) long, or, with
// swizzle_bytes == 0, unswizzled rows of any multiple of 16 bytes up to 256
// elements; out-of-bounds elements read as zero.
int tma_encode_2d(CUtensorMap* map, CUtensorMapDataType dt, int elem_bytes, const void* base,
                  uint64_t inner, uint64_t outer, uint64_t ld_elems, uint32_t box_inner,
                  uint32_t box_outer, int swizzle_bytes) {
  if (!tma_available()) return COMPAR_ERR_UNSUPPORTED;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0) return COMPAR_ERR_INVALID;
  if ((ld_elems * elem_bytes) % 16 != 0) return COMPAR_ERR_INVALID;
  if (swizzle_bytes == 0) {
    // unswizzled box: rows of box_inner elements, a multiple of 16 bytes
    if (box_inner == 0 || box_inner > 256 || (box_inner * elem_bytes) % 16 != 0 ||
        box_outer == 0 || box_outer > 256)
      return COMPAR_ERR_INVALID;
  } else if ((swizzle_bytes != 64 && swizzle_bytes != 128) ||
             box_inner * elem_bytes != static_cast<uint32_t>(swizzle_bytes) || box_outer == 0 ||
             box_outer > 256) {
    return COMPAR_ERR_INVALID;
  }
  MapKey key;
  memset(&key, 0, sizeof(key));  // padding bytes take part in the comparison
  key.base = reinterpret_cast<uintptr_t>(base);
  key.inner = inner;
  key.outer = outer;
  key.ld = ld_elems;
  key.box_inner = box_inner;
  key.box_outer = box_outer;
  key.dt = static_cast<int>(dt);
  key.elem = elem_bytes;
  key.swizzle = swizzle_bytes;
  {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    if (!g_cache) g_cache = new std::unordered_map<MapKey, CUtensorMap, MapKeyHash>();
    auto it = g_cache->find(key);
    if (it != g_cache->end()) {
      *map = it->second;
      return COMPAR_OK;
    }
  }
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {ld_elems * static_cast<uint64_t>(elem_bytes)};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = g_encode(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE,
                              swizzle_bytes == 128  ? CU_TENSOR_MAP_SWIZZLE_128B
                              : swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                    : CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return COMPAR_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_cache_mu);
  if (g_cache->size() >= kMapCacheMax) g_cache->clear();
  (*g_cache)[key] = *map;
  return COMPAR_OK;
}

}  // namespace compar
