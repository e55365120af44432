// Asynchronous-copy helpers for sm_103a: mbarriers in shared memory and
// TMA tile loads (cp.async.bulk.tensor) described by a CUtensorMap.  Every
// wait is bounded by kSpinLimit polls; a wait that gives up returns false
// and the caller records KS_ETIMEOUT.
#pragma once

#include <cuda.h>
#include <cstdint>

#include "ks_internal.cuh"

namespace ks {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}

// Make barrier initialisation visible to the async proxy (TMA).
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Arrive once and announce `bytes` of transactions for the current phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait_parity(uint64_t *bar, uint32_t parity) {
  const uint32_t a = smem_addr(bar);
  for (long long spins = 0; spins < kSpinLimit; ++spins) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n"
        "selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 4-D tile load of the box at coordinates (c0, c1, c2, c3) (c0 innermost)
// into shared memory; completion is signalled on `bar` as transaction bytes.
// c0 times the element size must be a multiple of 16 bytes; the other
// coordinates may lie outside the tensor (the box is then zero-filled).
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int c0, int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(c0), "r"(c1), "r"(c2),
      "r"(c3)
      : "memory");
}

// 2-D tile load (x innermost) into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%3, %4}], [%2];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(c0), "r"(c1)
      : "memory");
}

__device__ __forceinline__ void prefetch_tensor_map(const CUtensorMap *map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Host: a 4-D tiled tensor map over a dense row-major array with extents
// dims[0..3] (dims[0] innermost) of elem_bytes-byte elements, box extents
// box[0..3], zero fill outside the tensor.  Fails (KS_EINVAL) when the base
// address or a stride is not a multiple of 16 bytes, so callers can take
// their plain-load path instead.
ks_status encode_tensor_map_4d(CUtensorMap *map, const void *base, int elem_bytes,
                               const uint64_t dims[4], const uint32_t box[4]);

// Host: a 2-D FP32 tiled tensor map over a row-major rows x cols array
// (cols innermost, row pitch cols * 4 bytes), box {32, box_rows} with the
// 128-byte swizzle (the K-major layout the tensor cores read), zero fill
// outside the tensor.  KS_EINVAL when the base or the pitch is not a
// multiple of 16 bytes.
ks_status encode_tensor_map_2d_sw128(CUtensorMap *map, const float *base, uint64_t rows,
                                     uint64_t cols, uint32_t box_rows);

}  // namespace ks
