// Host side of the TMA helpers: tensor-map encoding through the driver
// entry point that the runtime hands out (no link against libcuda).
#include <cudaTypedefs.h>

#include <mutex>

#include "ks_async.cuh"

namespace ks {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

void load_encode() {
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  else
    cudaGetLastError();
}

}  // namespace

ks_status encode_tensor_map_4d(CUtensorMap *map, const void *base, int elem_bytes,
                               const uint64_t dims[4], const uint32_t box[4]) {
  std::call_once(g_encode_once, load_encode);
  if (!g_encode) return set_error(KS_EINVAL, "tensor-map encoder unavailable");
  if (reinterpret_cast<uintptr_t>(base) % 16 != 0)
    return set_error(KS_EINVAL, "tensor map: base address not 16-byte aligned");
  CUtensorMapDataType dt;
  if (elem_bytes == 4) dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  else if (elem_bytes == 8) dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  else return set_error(KS_EINVAL, "tensor map: unsupported element size");
  cuuint64_t gdim[4], gstride[3];
  cuuint32_t bdim[4], estride[4] = {1, 1, 1, 1};
  uint64_t s = (uint64_t)elem_bytes;
  for (int i = 0; i < 4; ++i) {
    gdim[i] = dims[i];
    bdim[i] = box[i];
    if (i > 0) {
      if (s % 16 != 0) return set_error(KS_EINVAL, "tensor map: stride not a multiple of 16 bytes");
      gstride[i - 1] = s;
    }
    s *= dims[i];
  }
  if ((uint64_t)box[0] * elem_bytes % 16 != 0)
    return set_error(KS_EINVAL, "tensor map: inner box not a multiple of 16 bytes");
  const CUresult r = g_encode(map, dt, 4, const_cast<void *>(base), gdim, gstride, bdim, estride,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(KS_EINVAL, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return KS_OK;
}

}  // namespace ks
