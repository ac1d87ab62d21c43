// TMA tensor-map encoding.  cuTensorMapEncodeTiled is a driver API call; it
// is resolved at run time through the runtime's driver entry-point query so
// the library does not link libcuda directly.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "common.h"

namespace compar {
namespace {

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
// whose rows are exactly one swizzle width (64 or 128 bytes) long;
// out-of-bounds elements read as zero.
int tma_encode_2d(CUtensorMap* map, CUtensorMapDataType dt, int elem_bytes, const void* base,
                  uint64_t inner, uint64_t outer, uint64_t ld_elems, uint32_t box_inner,
                  uint32_t box_outer, int swizzle_bytes) {
  if (!tma_available()) return COMPAR_ERR_UNSUPPORTED;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0) return COMPAR_ERR_INVALID;
  if ((ld_elems * elem_bytes) % 16 != 0) return COMPAR_ERR_INVALID;
  if ((swizzle_bytes != 64 && swizzle_bytes != 128) ||
      box_inner * elem_bytes != static_cast<uint32_t>(swizzle_bytes) || box_outer == 0 ||
      box_outer > 256)
    return COMPAR_ERR_INVALID;
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {ld_elems * static_cast<uint64_t>(elem_bytes)};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = g_encode(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE,
                              swizzle_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                                   : CU_TENSOR_MAP_SWIZZLE_64B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? COMPAR_OK : COMPAR_ERR_CUDA;
}

}  // namespace compar
