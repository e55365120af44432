// Tall-skinny Gram A^T B of the FP32 phase on the 5th-generation tensor
// cores (tcgen05, kind::tf32), accumulator in tensor memory.
//
// A (n x pa) and B (n x qb) are row-major FP32.  A block owns a 128 x 64
// output tile (columns a0.. of A, b0.. of B) and a chunk of rows; it stages
// 32 rows at a time into shared memory in the K-major core-matrix layout
// (8 rows x 16 bytes per core matrix, no swizzle), split into TF32 high and
// low parts (x = hi + lo, hi = x with the low 13 mantissa bits cleared), and
// one thread issues hi.hi + hi.lo + lo.hi products (3 x 4 MMAs of
// 128 x 64 x 8 per stage) into one FP32 accumulator in tensor memory.  Two
// stage buffers alternate; a stage buffer is refilled only after the MMAs
// that read it have committed to its mbarrier.  All waits are bounded: a
// block that waits too long records KS_ETIMEOUT and stops.  The chunk's
// 128 x 64 partial is read back with tcgen05.ld and written as FP64 partials
// that the caller sums in chunk order.
#include <cstdint>

#include "ks_device.cuh"

namespace ks {

namespace {

constexpr int kTcM = 128, kTcN = 64, kTcK = 32;   // tile rows, cols, rows per stage
constexpr int kTcThreads = 256;
constexpr int kTcCols = 64;                       // TMEM columns allocated
constexpr int kTileABytes = kTcM * kTcK * 4;      // 16 KiB
constexpr int kTileBBytes = kTcN * kTcK * 4;      //  8 KiB
constexpr int kStageBytes = 2 * kTileABytes + 2 * kTileBBytes;   // hi + lo of A and B
constexpr int kTcSmem = 2 * kStageBytes + 1024;   // two stages + alignment slack

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (r, k) of an R x 32 K-major tile: core matrices of
// 8 rows x 16 bytes, K-adjacent ones 128 bytes apart (LBO), row groups of 8
// 1024 bytes apart (SBO)
__device__ __forceinline__ int kmajor_offset(int r, int k) {
  return (r >> 3) * 1024 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4;
}

// shared-memory matrix descriptor: start address, LBO = 128 B, SBO = 1024 B,
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor: D FP32, A and B TF32, both K-major, N = 64, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                            ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
      :: "r"(tmem), "l"(da), "l"(db), "r"(kIdesc), "r"(acc));
}

// bounded wait for phase `parity` of the mbarrier; false when it gave up
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (long long spins = 0; spins < kSpinLimit; ++spins) {
    uint32_t done;
    asm volatile("{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n"
                 "selp.u32 %0, 1, 0, q;\n}\n" : "=r"(done) : "r"(mbar), "r"(parity));
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  lo = x - hi;
}

__global__ void __launch_bounds__(kTcThreads) gram_tc_kernel(long long n, int pa, int qb,
                                                            long long rows_per, int tiles_b,
                                                            const float *__restrict__ A,
                                                            const float *__restrict__ B,
                                                            double *__restrict__ part,
                                                            int *status) {
  extern __shared__ __align__(1024) unsigned char dyn_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)dyn_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int ta = blockIdx.x / tiles_b, tb = blockIdx.x % tiles_b;
  const int a0 = ta * kTcM, b0 = tb * kTcN;
  const int chunk = blockIdx.y;
  const long long r0 = chunk * rows_per;
  long long r1 = r0 + rows_per;
  if (r1 > n) r1 = n;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_slot)), "r"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&mbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&mbar[1])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;

  uint32_t phase[2] = {0u, 0u};
  int issued = 0;                       // stages issued so far
  bool failed = false;                  // block-uniform
  // only the valid columns of the tiles are staged each stage; the padding
  // rows of the K-major tiles are zeroed once in both stage buffers
  const int mw = min(kTcM, pa - a0), nw = min(kTcN, qb - b0);
  for (int t = tid; t < 2 * (kTcM * kTcK + kTcN * kTcK); t += kTcThreads) {
    const int b = t / (kTcM * kTcK + kTcN * kTcK);
    int e = t % (kTcM * kTcK + kTcN * kTcK);
    unsigned char *st = smem + b * kStageBytes;
    if (e < kTcM * kTcK) {
      const int k = e / kTcM, m = e % kTcM;
      if (m >= mw) {
        const int off = kmajor_offset(m, k);
        *(float *)(st + off) = 0.f;
        *(float *)(st + kTileABytes + off) = 0.f;
      }
    } else {
      e -= kTcM * kTcK;
      const int k = e / kTcN, c = e % kTcN;
      if (c >= nw) {
        const int off = kmajor_offset(c, k);
        *(float *)(st + 2 * kTileABytes + off) = 0.f;
        *(float *)(st + 2 * kTileABytes + kTileBBytes + off) = 0.f;
      }
    }
  }
  // register prefetch of one stage: A values (k, m < mw), B values (k, c < nw)
  constexpr int kRegA = kTcM * kTcK / kTcThreads, kRegB = kTcN * kTcK / kTcThreads;
  float ra[kRegA], rb[kRegB];
  auto fetch = [&](long long r) {
#pragma unroll
    for (int i = 0; i < kRegA; ++i) {
      const int t = tid + i * kTcThreads;
      const int k = t / mw, m = t - k * mw;
      const long long row = r + k;
      ra[i] = (k < kTcK && row < r1) ? A[row * pa + a0 + m] : 0.f;
    }
#pragma unroll
    for (int i = 0; i < kRegB; ++i) {
      const int t = tid + i * kTcThreads;
      const int k = t / nw, c = t - k * nw;
      const long long row = r + k;
      rb[i] = (k < kTcK && row < r1) ? B[row * qb + b0 + c] : 0.f;
    }
  };
  __syncthreads();
  if (r0 < r1) fetch(r0);
  for (long long r = r0; r < r1; r += kTcK, ++issued) {
    const int buf = issued & 1;
    unsigned char *st = smem + buf * kStageBytes;
    float *ah = (float *)st, *al = (float *)(st + kTileABytes);
    float *bh = (float *)(st + 2 * kTileABytes), *bl = (float *)(st + 2 * kTileABytes + kTileBBytes);
    // the buffer was last read by stage issued-2: wait for its commit
    if (issued >= 2) {
      int ok = 1;
      if (!mbar_wait(smem_u32(&mbar[buf]), phase[buf])) ok = 0;
      phase[buf] ^= 1u;
      if (!__syncthreads_and(ok)) {
        if (tid == 0) atomicCAS(status, 0, (int)KS_ETIMEOUT);
        failed = true;
        break;
      }
    }
#pragma unroll
    for (int i = 0; i < kRegA; ++i) {
      const int t = tid + i * kTcThreads;
      const int k = t / mw, m = t - k * mw;
      if (k < kTcK) {
        float hi, lo;
        split_tf32(ra[i], hi, lo);
        const int off = kmajor_offset(m, k);
        *(float *)((unsigned char *)ah + off) = hi;
        *(float *)((unsigned char *)al + off) = lo;
      }
    }
#pragma unroll
    for (int i = 0; i < kRegB; ++i) {
      const int t = tid + i * kTcThreads;
      const int k = t / nw, c = t - k * nw;
      if (k < kTcK) {
        float hi, lo;
        split_tf32(rb[i], hi, lo);
        const int off = kmajor_offset(c, k);
        *(float *)((unsigned char *)bh + off) = hi;
        *(float *)((unsigned char *)bl + off) = lo;
      }
    }
    // next stage's loads overlap this stage's MMAs
    if (r + kTcK < r1) fetch(r + kTcK);
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t sah = smem_u32(ah), sal = smem_u32(al), sbh = smem_u32(bh), sbl = smem_u32(bl);
#pragma unroll
      for (int ks = 0; ks < kTcK / 8; ++ks) {
        const uint32_t o = ks * 256;
        mma_tf32(tmem, smem_desc(sah + o), smem_desc(sbh + o), (issued > 0 || ks > 0) ? 1u : 0u);
        mma_tf32(tmem, smem_desc(sah + o), smem_desc(sbl + o), 1u);
        mma_tf32(tmem, smem_desc(sal + o), smem_desc(sbh + o), 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(smem_u32(&mbar[buf])));
    }
  }
  // drain: wait for the last one or two stages
  int ok = failed ? 0 : 1;
  if (ok && issued > 0) {
    const int last = (issued - 1) & 1;
    if (issued >= 2 && !mbar_wait(smem_u32(&mbar[last ^ 1]), phase[last ^ 1])) ok = 0;
    if (!mbar_wait(smem_u32(&mbar[last]), phase[last])) ok = 0;
  }
  ok = __syncthreads_and(ok);
  if (!ok && tid == 0 && !failed) atomicCAS(status, 0, (int)KS_ETIMEOUT);
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok && warp < 4) {
    uint32_t v[kTcN];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
        "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
        "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
          "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
          "=r"(v[31]), "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]),
          "=r"(v[37]), "=r"(v[38]), "=r"(v[39]), "=r"(v[40]), "=r"(v[41]), "=r"(v[42]),
          "=r"(v[43]), "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]), "=r"(v[48]),
          "=r"(v[49]), "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]),
          "=r"(v[55]), "=r"(v[56]), "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]),
          "=r"(v[61]), "=r"(v[62]), "=r"(v[63])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    const int arow = a0 + warp * 32 + (tid & 31);
    if (arow < pa) {
      double *dst = part + (long long)chunk * pa * qb + (long long)arow * qb;
      for (int j = 0; j < kTcN; ++j)
        if (b0 + j < qb) dst[b0 + j] = issued > 0 ? (double)__uint_as_float(v[j]) : 0.0;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTcCols));
}

// out = alpha (A1 C1 + A2 C2) + beta Bm on the tensor cores: a block owns
// 128 rows x 64 output columns; K runs over the columns of A1 then A2 in
// stages of 32.  The A rows are already K-major (row-major blocks); the C
// slices are transposed into the K-major layout.  Same 3 x TF32 split,
// double buffering and bounded waits as the Gram kernel.
__global__ void __launch_bounds__(kTcThreads) combine_tc_kernel(
    long long n, int q, const float *__restrict__ A1, int k1, const double *__restrict__ C1,
    const float *__restrict__ A2, int k2, const double *__restrict__ C2, float alpha, float beta,
    const float *__restrict__ Bm, float *__restrict__ out, int *status) {
  extern __shared__ __align__(1024) unsigned char dyn_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)dyn_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const long long row0 = (long long)blockIdx.x * kTcM;
  const int c0 = blockIdx.y * kTcN;
  const int K = k1 + (A2 ? k2 : 0);
  const int nw = min(kTcN, q - c0);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_slot)), "r"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&mbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&mbar[1])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;

  uint32_t phase[2] = {0u, 0u};
  int issued = 0;
  bool failed = false;
  for (int kb = 0; kb < K; kb += kTcK, ++issued) {
    const int buf = issued & 1;
    unsigned char *st = smem + buf * kStageBytes;
    float *ah = (float *)st, *al = (float *)(st + kTileABytes);
    float *bh = (float *)(st + 2 * kTileABytes), *bl = (float *)(st + 2 * kTileABytes + kTileBBytes);
    if (issued >= 2) {
      int ok = 1;
      if (!mbar_wait(smem_u32(&mbar[buf]), phase[buf])) ok = 0;
      phase[buf] ^= 1u;
      if (!__syncthreads_and(ok)) {
        if (tid == 0) atomicCAS(status, 0, (int)KS_ETIMEOUT);
        failed = true;
        break;
      }
    }
    // A slice: rows row0.., K columns kb..kb+31 (k-contiguous in memory)
    for (int t = tid; t < kTcM * kTcK; t += kTcThreads) {
      const int m = t / kTcK, k = t % kTcK;
      const long long row = row0 + m;
      const int kk = kb + k;
      float x = 0.f;
      if (row < n && kk < K) x = kk < k1 ? A1[row * k1 + kk] : A2[row * k2 + (kk - k1)];
      float hi, lo;
      split_tf32(x, hi, lo);
      const int off = kmajor_offset(m, k);
      *(float *)((unsigned char *)ah + off) = hi;
      *(float *)((unsigned char *)al + off) = lo;
    }
    // C slice transposed: element (c, k) = C[kb + k][c0 + c]
    for (int t = tid; t < kTcN * kTcK; t += kTcThreads) {
      const int k = t / kTcN, c = t % kTcN;
      const int kk = kb + k;
      float x = 0.f;
      if (c < nw && kk < K)
        x = (float)(kk < k1 ? C1[(long long)kk * q + c0 + c] : C2[(long long)(kk - k1) * q + c0 + c]);
      float hi, lo;
      split_tf32(x, hi, lo);
      const int off = kmajor_offset(c, k);
      *(float *)((unsigned char *)bh + off) = hi;
      *(float *)((unsigned char *)bl + off) = lo;
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t sah = smem_u32(ah), sal = smem_u32(al), sbh = smem_u32(bh), sbl = smem_u32(bl);
#pragma unroll
      for (int ks = 0; ks < kTcK / 8; ++ks) {
        const uint32_t o = ks * 256;
        mma_tf32(tmem, smem_desc(sah + o), smem_desc(sbh + o), (issued > 0 || ks > 0) ? 1u : 0u);
        mma_tf32(tmem, smem_desc(sah + o), smem_desc(sbl + o), 1u);
        mma_tf32(tmem, smem_desc(sal + o), smem_desc(sbh + o), 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(smem_u32(&mbar[buf])));
    }
  }
  int ok = failed ? 0 : 1;
  if (ok && issued > 0) {
    const int last = (issued - 1) & 1;
    if (issued >= 2 && !mbar_wait(smem_u32(&mbar[last ^ 1]), phase[last ^ 1])) ok = 0;
    if (!mbar_wait(smem_u32(&mbar[last]), phase[last])) ok = 0;
  }
  ok = __syncthreads_and(ok);
  if (!ok && tid == 0 && !failed) atomicCAS(status, 0, (int)KS_ETIMEOUT);
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok && warp < 4) {
    uint32_t v[kTcN];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
        "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
        "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
          "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
          "=r"(v[31]), "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]),
          "=r"(v[37]), "=r"(v[38]), "=r"(v[39]), "=r"(v[40]), "=r"(v[41]), "=r"(v[42]),
          "=r"(v[43]), "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]), "=r"(v[48]),
          "=r"(v[49]), "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]),
          "=r"(v[55]), "=r"(v[56]), "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]),
          "=r"(v[61]), "=r"(v[62]), "=r"(v[63])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    const long long row = row0 + warp * 32 + (tid & 31);
    if (row < n) {
      float *dst = out + row * q + c0;
      const float *bm = Bm ? Bm + row * q + c0 : nullptr;
      for (int j = 0; j < nw; ++j) {
        float y = alpha * __uint_as_float(v[j]);
        if (bm) y = fmaf(beta, bm[j], y);
        dst[j] = y;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTcCols));
}

}  // namespace

ks_status configure_tc_kernels() {
  KS_CUDA_TRY(cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   kTcSmem));
  KS_CUDA_TRY(cudaFuncSetAttribute(combine_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   kTcSmem));
  return KS_OK;
}

ks_status launch_combine_tc(Problem &P, const float *A1, int k1, const double *C1,
                            const float *A2, int k2, const double *C2, double alpha, double beta,
                            const float *Bm, float *out, int q) {
  dim3 grid((unsigned)((P.n + kTcM - 1) / kTcM), (unsigned)((q + kTcN - 1) / kTcN));
  const int K = k1 + (A2 ? k2 : 0);
  {
    ProfScope ps_(P.stream, KP_COMBINE, 2.0 * P.n * q * K,
                  (double)P.n * (K + q * (Bm ? 2 : 1)) * sizeof(float));
    combine_tc_kernel<<<grid, kTcThreads, kTcSmem, P.stream>>>(P.n, q, A1, k1, C1, A2, k2, C2,
                                                               (float)alpha, (float)beta, Bm, out,
                                                               P.dstatus);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

// Chunks of the tensor-core Gram: about two blocks per SM over all tiles,
// at least 512 rows per chunk.
int gram_tc_chunks(const Problem &P, int pa, int qb) {
  const int tiles = ((pa + kTcM - 1) / kTcM) * ((qb + kTcN - 1) / kTcN);
  int chunks = (2 * P.sms + tiles - 1) / tiles;
  const int maxc = (P.n + 511) / 512;
  if (chunks > maxc) chunks = maxc;
  if (chunks < 1) chunks = 1;
  return chunks;
}

ks_status launch_gram_tc(Problem &P, const float *A, int pa, const float *B, int qb,
                         double *part, int chunks) {
  const int tiles_a = (pa + kTcM - 1) / kTcM, tiles_b = (qb + kTcN - 1) / kTcN;
  long long rows_per = (P.n + chunks - 1) / chunks;
  rows_per = (rows_per + kTcK - 1) / kTcK * kTcK;
  {
    ProfScope ps_(P.stream, KP_GRAM, 2.0 * P.n * pa * qb, (double)P.n * (pa + qb) * sizeof(float));
    gram_tc_kernel<<<dim3(tiles_a * tiles_b, chunks), kTcThreads, kTcSmem, P.stream>>>(
        P.n, pa, qb, rows_per, tiles_b, A, B, part, P.dstatus);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

}  // namespace ks
