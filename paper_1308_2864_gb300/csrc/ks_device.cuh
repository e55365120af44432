// Device helpers: deterministic block reductions, a bounded software grid
// barrier for cooperative launches, and uncached loads for data that other
// blocks of the same launch have written.
#pragma once

#include <cuda_runtime.h>

#include "ks_internal.cuh"

namespace ks {

// ---------------------------------------------------------------- bounds-checked build
// Compiled with -DKS_DEBUG_BOUNDS, KS_IN(i, len) checks a computed index
// before the access it guards: an index outside [0, len) is counted, with
// the source line of the first one, in this translation unit's device
// counters, and the guarded access is skipped, so the kernel runs on and the
// host reads the record through ks_debug_bounds (no trap, no fault).
// Without the macro KS_IN is `true` and costs nothing.
#ifdef KS_DEBUG_BOUNDS
namespace {
__device__ unsigned long long oob_count;
__device__ int oob_first_line;

__device__ __noinline__ bool oob_note(int line) {
  if (atomicAdd(&oob_count, 1ull) == 0ull) oob_first_line = line;
  return false;
}

// this translation unit's record, then cleared
[[maybe_unused]] void oob_collect(unsigned long long *count, int *line) {
  unsigned long long c = 0;
  int l = 0;
  cudaDeviceSynchronize();
  cudaMemcpyFromSymbol(&c, oob_count, sizeof(c));
  cudaMemcpyFromSymbol(&l, oob_first_line, sizeof(l));
  const unsigned long long zc = 0;
  const int zl = 0;
  cudaMemcpyToSymbol(oob_count, &zc, sizeof(zc));
  cudaMemcpyToSymbol(oob_first_line, &zl, sizeof(zl));
  *count = c;
  *line = l;
}
}  // namespace
#define KS_IN(i, len) \
  ((unsigned long long)(long long)(i) < (unsigned long long)(long long)(len) ? true \
                                                                            : ks::oob_note(__LINE__))
#define KS_OOB_READER(name) \
  void oob_read_##name(unsigned long long *c, int *l) { oob_collect(c, l); }
#else
#define KS_IN(i, len) true
#define KS_OOB_READER(name)
#endif

__device__ __forceinline__ double ldcg(const double *p) { return __ldcg(p); }

// Sum over a block of blockDim.x (a multiple of 32, <= 1024) threads in a
// fixed order: xor-butterfly inside each warp, then warp 0 adds the warp
// sums in the same butterfly.  Every thread receives the result.
__device__ __forceinline__ double block_sum(double v, double *smem /* >= 33 */) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) smem[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double w = lane < nw ? smem[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (lane == 0) smem[32] = w;
  }
  __syncthreads();
  double r = smem[32];
  __syncthreads();
  return r;
}

// Sum nb values src[0..nb) in a fixed order by the whole block (strided
// partial sums in index order, then block_sum).  src may have been written
// by other blocks of this launch, so it is read through L2.
__device__ __forceinline__ double block_sum_array(const double *src, int nb, double *smem) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += ldcg(src + i);
  return block_sum(acc, smem);
}

// Last-block reduction: every block has written its nchan partial sums to
// part[c * nb + blockIdx.x] (thread 0); the block that arrives last sums
// each channel over all blocks in index order (the same order whichever
// block is last, so the result is deterministic), writes scale * sum to
// out[c] and re-arms the counter for the next launch on the stream.
__device__ __forceinline__ void grid_reduce_tail(const double *part, int nb, int nchan,
                                                 double *out, double scale,
                                                 unsigned int *counter, double *smem) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    s_last = (prev == (unsigned int)nb - 1u);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int c = 0; c < nchan; ++c) {
    const double sacc = block_sum_array(part + (long long)c * nb, nb, smem);
    if (threadIdx.x == 0) out[c] = scale * sacc;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// Polls of a grid-barrier wait before the waiting thread starts to sleep.
constexpr long long kSpinFree = 1 << 14;

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int *p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Barrier of the nb blocks that share `bar` inside a cooperative launch (all
// blocks of the launch co-resident; nb = the whole grid, or the blocks of one
// system in a batched launch).
// Every wait is bounded: a block that spins longer than kSpinLimit records
// KS_ETIMEOUT in *status and leaves the barrier.  Returns false when the
// status word holds an error, so that callers can return together.
__device__ __forceinline__ bool grid_barrier_n(GridBarrier *bar, int *status, unsigned int nb) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int gen = ld_acquire_gpu(&bar->gen);
    __threadfence();
    const unsigned int arrived = atomicAdd(&bar->count, 1u);
    if (arrived == nb - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      // poll without sleeping first (a barrier between short phases is
      // usually released within a few microseconds), then back off
      long long spins = 0;
      unsigned int ns = 32;
      while (ld_acquire_gpu(&bar->gen) == gen) {
        if (++spins > kSpinLimit) {
          atomicCAS(status, 0, (int)KS_ETIMEOUT);
          break;
        }
        if (spins > kSpinFree) {
          __nanosleep(ns);
          if (ns < 256) ns <<= 1;
        }
      }
    }
    __threadfence();
    s_ok = (*(volatile int *)status == 0);
  }
  __syncthreads();
  return s_ok != 0;
}

// The same over the whole grid of the launch.
__device__ __forceinline__ bool grid_barrier(GridBarrier *bar, int *status) {
  return grid_barrier_n(bar, status, gridDim.x * gridDim.y * gridDim.z);
}

// 27-point Q1 stencil coefficient classes (see the stiffness/mass
// construction in ks_stencil.cu): centre, face (6), edge (12), corner (8).
struct StencilCoef {
  double k0, kf, ke, kc;  // stiffness
  double m0, mf, me, mc;  // mass
};

__host__ __device__ inline StencilCoef q1_coefficients(double h) {
  // 1-D entries: K1 = (1/h)[-1, 2, -1], M1 = (h/6)[1, 4, 1]; the 3-D
  // coefficient at an offset with j nonzero components is a sum of products
  // of these (K = K1 M1 M1 + M1 K1 M1 + M1 M1 K1, M = M1 M1 M1).
  const double k_0 = 2.0 / h, k_1 = -1.0 / h;
  const double m_0 = 4.0 * h / 6.0, m_1 = h / 6.0;
  StencilCoef c;
  c.k0 = 3.0 * k_0 * m_0 * m_0;
  c.kf = k_1 * m_0 * m_0 + 2.0 * m_1 * k_0 * m_0;
  c.ke = 2.0 * k_1 * m_1 * m_0 + m_1 * m_1 * k_0;
  c.kc = 3.0 * k_1 * m_1 * m_1;
  c.m0 = m_0 * m_0 * m_0;
  c.mf = m_1 * m_0 * m_0;
  c.me = m_1 * m_1 * m_0;
  c.mc = m_1 * m_1 * m_1;
  return c;
}

}  // namespace ks
