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

// Encoded maps by (base, element size, dims, box): a map holds only the
// address and the layout, so a cached one is exact for any allocation that
// occupies the same address with the same layout.  The iteration re-uses a
// few blocks over and over, and encoding runs through the driver, so the
// launches of a solve find their maps here.
struct MapKey {
  const void *base;
  int elem;                 // element bytes; negative: the 2-D 128-byte-swizzled form
  uint64_t dims[4];
  uint32_t box[4];
  bool operator==(const MapKey &o) const {
    if (base != o.base || elem != o.elem) return false;
    for (int i = 0; i < 4; ++i)
      if (dims[i] != o.dims[i] || box[i] != o.box[i]) return false;
    return true;
  }
};

constexpr int kMapCache = 64;
struct MapCache {
  std::mutex mu;
  MapKey key[kMapCache];
  CUtensorMap map[kMapCache];
  unsigned long long used[kMapCache] = {};
  unsigned long long tick = 0;
  int n = 0;
};
MapCache g_maps;

ks_status encode_uncached(CUtensorMap *map, const void *base, int elem_bytes,
                          const uint64_t dims[4], const uint32_t box[4]);
ks_status encode_sw128_uncached(CUtensorMap *map, const float *base, uint64_t rows,
                                uint64_t cols, uint32_t box_rows);

// Look up key k; on a miss encode with `make` and remember the result.
template <typename F>
ks_status cached_map(const MapKey &k, CUtensorMap *map, F make) {
  std::lock_guard<std::mutex> lock(g_maps.mu);
  for (int i = 0; i < g_maps.n; ++i)
    if (g_maps.key[i] == k) {
      g_maps.used[i] = ++g_maps.tick;
      *map = g_maps.map[i];
      return KS_OK;
    }
  KS_TRY(make());
  int slot = 0;
  if (g_maps.n < kMapCache) {
    slot = g_maps.n++;
  } else {
    for (int i = 1; i < kMapCache; ++i)     // least recently used
      if (g_maps.used[i] < g_maps.used[slot]) slot = i;
  }
  g_maps.key[slot] = k;
  g_maps.map[slot] = *map;
  g_maps.used[slot] = ++g_maps.tick;
  return KS_OK;
}

}  // namespace

ks_status encode_tensor_map_4d(CUtensorMap *map, const void *base, int elem_bytes,
                               const uint64_t dims[4], const uint32_t box[4]) {
  const MapKey k{base, elem_bytes, {dims[0], dims[1], dims[2], dims[3]},
                 {box[0], box[1], box[2], box[3]}};
  return cached_map(k, map, [&] { return encode_uncached(map, base, elem_bytes, dims, box); });
}

ks_status encode_tensor_map_2d_sw128(CUtensorMap *map, const float *base, uint64_t rows,
                                     uint64_t cols, uint32_t box_rows) {
  const MapKey k{base, -4, {cols, rows, 0, 0}, {32u, box_rows, 0, 0}};
  return cached_map(k, map,
                    [&] { return encode_sw128_uncached(map, base, rows, cols, box_rows); });
}

namespace {

ks_status encode_uncached(CUtensorMap *map, const void *base, int elem_bytes,
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

ks_status encode_sw128_uncached(CUtensorMap *map, const float *base, uint64_t rows,
                                uint64_t cols, uint32_t box_rows) {
  std::call_once(g_encode_once, load_encode);
  if (!g_encode) return set_error(KS_EINVAL, "tensor-map encoder unavailable");
  if (reinterpret_cast<uintptr_t>(base) % 16 != 0 || (cols * 4) % 16 != 0)
    return set_error(KS_EINVAL, "tensor map: base or row pitch not a multiple of 16 bytes");
  cuuint64_t gdim[2] = {cols, rows};
  cuuint64_t gstride[1] = {cols * 4};
  cuuint32_t bdim[2] = {32u, box_rows}, estride[2] = {1, 1};
  const CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base),
                              gdim, gstride, bdim, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(KS_EINVAL, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return KS_OK;
}

}  // namespace

}  // namespace ks
